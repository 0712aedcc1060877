// The extern "C" boundary of libqsw.so (declared in include/qsw.h): argument
// validation, object lifetime and error translation.  All arithmetic of the
// path runs in the kernels of graph.cu, assemble.cu, norms.cu and series.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <exception>
#include <memory>
#include <new>

#include "op.h"
#include "params.cuh"

using qsw::Error;
using qsw::Op;

std::atomic<long long> qsw::g_launches{0};
std::atomic<long long> qsw::g_device_allocs{0};

namespace {

thread_local std::string g_orphan_error;

template <class F>
qsw_status guarded(qsw_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->last_error.clear();
    return QSW_OK;
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.msg;
    else g_orphan_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    return QSW_ERR_OOM;
  } catch (const std::exception& e) {
    if (ctx) ctx->last_error = e.what();
    return QSW_ERR_INVALID_ARG;
  }
}

void set_device(const qsw_ctx* ctx) {
  QSW_CUDA_TRY(cudaSetDevice(ctx->device));
  qsw::current_stream() = ctx->stream;
}

// Structural checks of a host CSR (see qsw.h conventions).
void check_csr(const qsw_csr* m, const char* name, bool allow_diag) {
  const std::string nm(name);
  QSW_CHECK_ARG(m != nullptr, QSW_ERR_INVALID_ARG, nm + " is NULL");
  QSW_CHECK_ARG(m->n >= 1, QSW_ERR_INVALID_ARG, nm + ".n must be >= 1");
  QSW_CHECK_ARG(m->nnz >= 0, QSW_ERR_INVALID_ARG, nm + ".nnz must be >= 0");
  QSW_CHECK_ARG(m->rowptr != nullptr, QSW_ERR_INVALID_ARG, nm + ".rowptr is NULL");
  QSW_CHECK_ARG(m->nnz == 0 || (m->col && m->w), QSW_ERR_INVALID_ARG, nm + ".col/.w is NULL");
  QSW_CHECK_ARG(m->rowptr[0] == 0 && m->rowptr[m->n] == m->nnz, QSW_ERR_INVALID_ARG,
                nm + ".rowptr must start at 0 and end at nnz");
  for (int i = 0; i < m->n; ++i) {
    QSW_CHECK_ARG(m->rowptr[i] <= m->rowptr[i + 1], QSW_ERR_INVALID_ARG,
                  nm + ".rowptr is not non-decreasing");
    for (int e = m->rowptr[i]; e < m->rowptr[i + 1]; ++e) {
      const int c = m->col[e];
      QSW_CHECK_ARG(c >= 0 && c < m->n, QSW_ERR_INVALID_ARG, nm + ": column index out of range");
      QSW_CHECK_ARG(e == m->rowptr[i] || m->col[e - 1] < c, QSW_ERR_INVALID_ARG,
                    nm + ": columns must be strictly increasing within a row");
      QSW_CHECK_ARG(isfinite(m->w[e]), QSW_ERR_INVALID_ARG, nm + ": non-finite value");
      if (!allow_diag)
        QSW_CHECK_ARG(c != i, QSW_ERR_NOT_SIMPLE, nm + ": self-loop (only simple graphs, Tr G = 0)");
    }
  }
}

double lookup(const qsw_csr* m, int i, int j, bool* found) {
  const int* b = m->col + m->rowptr[i];
  const int* e = m->col + m->rowptr[i + 1];
  const int* p = std::lower_bound(b, e, j);
  *found = p != e && *p == j;
  return *found ? m->w[p - m->col] : 0.0;
}

void check_ports(const qsw_port* p, int count, int N, const char* name) {
  QSW_CHECK_ARG(count >= 0 && count <= qsw::kMaxPorts, QSW_ERR_INVALID_ARG,
                std::string(name) + ": bad count");
  QSW_CHECK_ARG(count == 0 || p != nullptr, QSW_ERR_INVALID_ARG, std::string(name) + " is NULL");
  for (int k = 0; k < count; ++k) {
    QSW_CHECK_ARG(p[k].vertex >= 0 && p[k].vertex < N, QSW_ERR_INVALID_ARG,
                  std::string(name) + ": vertex out of range");
    QSW_CHECK_ARG(isfinite(p[k].rate) && p[k].rate > 0.0, QSW_ERR_INVALID_ARG,
                  std::string(name) + ": rate must be finite and > 0");
  }
}

// A complex host CSR (qsw_zcsr) as a ZMat, with the structural checks of
// check_csr; `hermitian` also requires A = A^dag.
qsw::ZMat zmat_of(const qsw_zcsr* m, int n, const char* name, bool hermitian) {
  const std::string nm(name);
  QSW_CHECK_ARG(m != nullptr, QSW_ERR_INVALID_ARG, nm + " is NULL");
  QSW_CHECK_ARG(m->n == n, QSW_ERR_INVALID_ARG, nm + " must be N x N");
  QSW_CHECK_ARG(m->nnz >= 0 && m->rowptr != nullptr, QSW_ERR_INVALID_ARG, nm + ": bad nnz/rowptr");
  QSW_CHECK_ARG(m->nnz == 0 || (m->col && m->re), QSW_ERR_INVALID_ARG, nm + ".col/.re is NULL");
  QSW_CHECK_ARG(m->rowptr[0] == 0 && m->rowptr[n] == m->nnz, QSW_ERR_INVALID_ARG,
                nm + ".rowptr must start at 0 and end at nnz");
  qsw::ZMat z;
  z.n = n;
  z.rowptr.assign(m->rowptr, m->rowptr + n + 1);
  for (int i = 0; i < n; ++i) {
    QSW_CHECK_ARG(m->rowptr[i] <= m->rowptr[i + 1], QSW_ERR_INVALID_ARG,
                  nm + ".rowptr is not non-decreasing");
    for (int e = m->rowptr[i]; e < m->rowptr[i + 1]; ++e) {
      const int c = m->col[e];
      QSW_CHECK_ARG(c >= 0 && c < n, QSW_ERR_INVALID_ARG, nm + ": column index out of range");
      QSW_CHECK_ARG(e == m->rowptr[i] || m->col[e - 1] < c, QSW_ERR_INVALID_ARG,
                    nm + ": columns must be strictly increasing within a row");
      const double im = m->im ? m->im[e] : 0.0;
      QSW_CHECK_ARG(isfinite(m->re[e]) && isfinite(im), QSW_ERR_INVALID_ARG, nm + ": non-finite value");
      z.col.push_back(c);
      z.val.push_back(std::complex<double>(m->re[e], im));
    }
  }
  if (hermitian)
    for (int i = 0; i < n; ++i)
      for (int e = z.rowptr[i]; e < z.rowptr[i + 1]; ++e) {
        const int j = z.col[e];
        const int* b = z.col.data() + z.rowptr[j];
        const int* f = z.col.data() + z.rowptr[j + 1];
        const int* q = std::lower_bound(b, f, i);
        QSW_CHECK_ARG(q != f && *q == i && z.val[q - z.col.data()] == std::conj(z.val[e]),
                      QSW_ERR_NOT_HERMITIAN, nm + " must be Hermitian");
      }
  return z;
}

// trans(1, G^u): the Laplacian of the undirected companion, G^u = max(G, G^T)
qsw::ZMat laplacian_undirected(const qsw_csr* G) {
  const int n = G->n;
  std::vector<std::vector<std::pair<int, double>>> rows(n);
  for (int i = 0; i < n; ++i)
    for (int e = G->rowptr[i]; e < G->rowptr[i + 1]; ++e) {
      rows[i].push_back({G->col[e], G->w[e]});
      rows[G->col[e]].push_back({i, G->w[e]});
    }
  qsw::ZMat L;
  L.n = n;
  L.rowptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    auto& r = rows[i];
    std::sort(r.begin(), r.end());
    std::vector<std::pair<int, double>> u;   // max over the two directions
    for (auto& e : r) {
      if (!u.empty() && u.back().first == e.first) u.back().second = std::max(u.back().second, e.second);
      else u.push_back(e);
    }
    double deg = 0.0;
    for (auto& e : u) deg += e.second;
    bool placed = false;
    for (auto& e : u) {
      if (!placed && e.first > i) {
        L.col.push_back(i);
        L.val.push_back(deg);
        placed = true;
      }
      L.col.push_back(e.first);
      L.val.push_back(-e.second);
    }
    if (!placed) {
      L.col.push_back(i);
      L.val.push_back(deg);
    }
    L.rowptr[i + 1] = (int)L.col.size();
  }
  return L;
}

qsw::ZMat zmat_of_real(const qsw_csr* G) {
  qsw::ZMat z;
  z.n = G->n;
  z.rowptr.assign(G->rowptr, G->rowptr + G->n + 1);
  z.col.assign(G->col, G->col + G->nnz);
  for (int e = 0; e < G->nnz; ++e) z.val.push_back(G->w[e]);
  return z;
}

void rebuild(Op& op, bool defer_norms) {
  if (op.gq.active) {   // global-interaction walk: matrix-free only
    qsw::build_global(op);
    op.norms_ready = !defer_norms;
    if (!defer_norms) qsw::compute_norms(op, nullptr, nullptr);
    return;
  }
  qsw::build_jumps(op);
  qsw::prep_matfree(op);
  op.L = qsw::Csr{};
  op.sell = qsw::Sell{};   // its values follow L: rebuilt by the next series that uses it
  op.norms_ready = !defer_norms;
  if (op.opkind == QSW_OPERATOR_CSR) {
    qsw::Csr LH;
    qsw::assemble(op, false, op.L);
    qsw::assemble(op, true, LH);
    qsw::compute_norms(op, &op.L, &LH);
    LH = qsw::Csr{};
    if (op.precision == QSW_C64_BULK) qsw::to_fp32(op, op.L);
    // the length heuristic until the first series tunes it (kept across
    // set_omega: the structure does not change)
    if (!op.tpr_fixed || op.tpr <= 0) op.tpr = qsw::choose_tpr((double)op.L.nnz / (double)op.n);
  } else if (!defer_norms) {
    qsw::compute_norms(op, nullptr, nullptr);
  }
}

void ensure_norms(Op& op) {
  if (op.norms_ready) return;
  qsw::compute_norms(op, nullptr, nullptr);
  op.norms_ready = true;
}

}  // namespace

extern "C" {

qsw_status qsw_create(qsw_ctx** out, int device, void* stream) {
  return guarded(nullptr, [&] {
    QSW_CHECK_ARG(out != nullptr, QSW_ERR_INVALID_ARG, "ctx is NULL");
    *out = nullptr;
    int count = 0;
    QSW_CUDA_TRY(cudaGetDeviceCount(&count));
    QSW_CHECK_ARG(device >= 0 && device < count, QSW_ERR_INVALID_ARG, "no such CUDA device");
    QSW_CUDA_TRY(cudaSetDevice(device));
    // keep freed device memory in the pool (stream-ordered reuse, no OS round trips)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      unsigned long long keep = ~0ULL;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    qsw_ctx* c = new qsw_ctx();
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
      delete c;
      QSW_CUDA_TRY(e);
    }
    try {
      qsw::upload_theta(device);
    } catch (...) {
      delete c;
      throw;
    }
    *out = c;
  });
}

void qsw_destroy(qsw_ctx* ctx) {
  if (ctx && ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx && ctx->copy) cudaStreamDestroy(ctx->copy);
  if (ctx && ctx->count_h) cudaFreeHost(ctx->count_h);
  delete ctx;
}

const char* qsw_last_error(const qsw_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_orphan_error.c_str();
}

qsw_status qsw_build_superoperator(qsw_ctx* ctx, const qsw_csr* G, const qsw_csr* H, double omega,
                                   const qsw_port* sources, int32_t n_sources,
                                   const qsw_port* sinks, int32_t n_sinks, int32_t precision,
                                   int32_t operator_kind, qsw_op** out) {
  return guarded(ctx, [&] {
    QSW_CHECK_ARG(ctx != nullptr && out != nullptr, QSW_ERR_INVALID_ARG, "ctx/out is NULL");
    *out = nullptr;
    check_csr(G, "G", false);
    for (int e = 0; e < G->nnz; ++e)
      QSW_CHECK_ARG(G->w[e] > 0.0, QSW_ERR_NOT_SIMPLE, "G: arc weights must be > 0");
    QSW_CHECK_ARG(isfinite(omega) && omega >= 0.0 && omega <= 1.0, QSW_ERR_OMEGA_RANGE,
                  "omega must lie in [0, 1]");
    QSW_CHECK_ARG(precision == QSW_C128 || precision == QSW_C64_BULK, QSW_ERR_INVALID_ARG,
                  "unknown precision");
    const bool defer = (operator_kind & QSW_BUILD_DEFER_NORMS) != 0;
    const bool fixed_schedule = (operator_kind & QSW_BUILD_FIXED_SCHEDULE) != 0;
    const bool rank64 = (operator_kind & QSW_BUILD_FP64_RANKING) != 0;
    operator_kind &= ~(QSW_BUILD_DEFER_NORMS | QSW_BUILD_FIXED_SCHEDULE | QSW_BUILD_FP64_RANKING);
    QSW_CHECK_ARG(operator_kind == QSW_OPERATOR_MATRIX_FREE || operator_kind == QSW_OPERATOR_CSR,
                  QSW_ERR_INVALID_ARG, "unknown operator kind");
    QSW_CHECK_ARG(!defer || operator_kind == QSW_OPERATOR_MATRIX_FREE, QSW_ERR_INVALID_ARG,
                  "deferred norms need the matrix-free operator");
    if (H) {
      check_csr(H, "H", true);
      QSW_CHECK_ARG(H->n == G->n, QSW_ERR_INVALID_ARG, "H must be N x N");
      for (int i = 0; i < H->n; ++i)
        for (int e = H->rowptr[i]; e < H->rowptr[i + 1]; ++e) {
          bool f = false;
          const double v = lookup(H, H->col[e], i, &f);
          QSW_CHECK_ARG(f && v == H->w[e], QSW_ERR_NOT_HERMITIAN, "H must be symmetric");
        }
    }
    check_ports(sources, n_sources, G->n, "sources");
    check_ports(sinks, n_sinks, G->n, "sinks");
    const long long Nt = (long long)G->n + n_sources + n_sinks;
    QSW_CHECK_ARG(Nt * Nt < (1LL << 31) - 1, QSW_ERR_TOO_LARGE,
                  "N~^2 does not fit 32-bit indices");
    set_device(ctx);

    std::unique_ptr<Op> op(new Op());
    op->ctx = ctx;
    op->precision = precision;
    op->opkind = operator_kind;
    if (fixed_schedule) {   // keep the length heuristic's lanes per row
      op->tpr_fixed = true;
      op->tpr = 0;
    }
    op->rank64 = rank64;
    op->omega = omega;
    op->N = G->n;
    op->Nt = (int)Nt;
    op->n = Nt * Nt;
    op->g_rowptr.assign(G->rowptr, G->rowptr + G->n + 1);
    op->g_col.assign(G->col, G->col + G->nnz);
    op->g_w.assign(G->w, G->w + G->nnz);
    if (H) {
      op->h_given = true;
      op->h_rowptr.assign(H->rowptr, H->rowptr + H->n + 1);
      op->h_col.assign(H->col, H->col + H->nnz);
      op->h_w.assign(H->w, H->w + H->nnz);
    }
    for (int k = 0; k < n_sources; ++k) {
      op->src_v.push_back(sources[k].vertex);
      op->src_r.push_back(sources[k].rate);
    }
    for (int k = 0; k < n_sinks; ++k) {
      op->snk_v.push_back(sinks[k].vertex);
      op->snk_r.push_back(sinks[k].rate);
    }
    qsw::build_graph(*op);
    rebuild(*op, defer);
    *out = reinterpret_cast<qsw_op*>(op.release());
  });
}

qsw_status qsw_build_global(qsw_ctx* ctx, int32_t n_vertices, const qsw_zcsr* H,
                            const qsw_zcsr* Ls, int32_t n_L, const qsw_zcsr* H_rot, double omega,
                            const qsw_port* sources, int32_t n_sources, const qsw_port* sinks,
                            int32_t n_sinks, int32_t precision, int32_t flags, qsw_op** out) {
  return guarded(ctx, [&] {
    QSW_CHECK_ARG(ctx != nullptr && out != nullptr, QSW_ERR_INVALID_ARG, "ctx/out is NULL");
    *out = nullptr;
    QSW_CHECK_ARG(n_vertices >= 1, QSW_ERR_INVALID_ARG, "n_vertices must be >= 1");
    QSW_CHECK_ARG(n_L >= 0 && n_L <= qsw::kMaxGlobalOps && (n_L == 0 || Ls), QSW_ERR_INVALID_ARG,
                  "n_L must be 0.." + std::to_string(qsw::kMaxGlobalOps));
    QSW_CHECK_ARG(isfinite(omega) && omega >= 0.0 && omega <= 1.0, QSW_ERR_OMEGA_RANGE,
                  "omega must lie in [0, 1]");
    QSW_CHECK_ARG(precision == QSW_C128 || precision == QSW_C64_BULK, QSW_ERR_INVALID_ARG,
                  "unknown precision");
    QSW_CHECK_ARG((flags & ~QSW_BUILD_DEFER_NORMS) == 0, QSW_ERR_INVALID_ARG, "unknown flags");
    check_ports(sources, n_sources, n_vertices, "sources");
    check_ports(sinks, n_sinks, n_vertices, "sinks");
    const long long Nt = (long long)n_vertices + n_sources + n_sinks;
    QSW_CHECK_ARG(Nt * Nt < (1LL << 31) - 1, QSW_ERR_TOO_LARGE, "N~^2 does not fit 32-bit indices");
    std::unique_ptr<Op> op(new Op());
    op->gq.H = zmat_of(H, n_vertices, "H", true);
    for (int k = 0; k < n_L; ++k)
      op->gq.Ls.push_back(zmat_of(&Ls[k], n_vertices, "L", false));
    if (H_rot) op->gq.Hrot = zmat_of(H_rot, n_vertices, "H_rot", true);
    set_device(ctx);
    op->gq.active = true;
    op->ctx = ctx;
    op->precision = precision;
    op->opkind = QSW_OPERATOR_MATRIX_FREE;
    op->omega = omega;
    op->N = n_vertices;
    op->Nt = (int)Nt;
    op->n = Nt * Nt;
    for (int k = 0; k < n_sources; ++k) {
      op->src_v.push_back(sources[k].vertex);
      op->src_r.push_back(sources[k].rate);
    }
    for (int k = 0; k < n_sinks; ++k) {
      op->snk_v.push_back(sinks[k].vertex);
      op->snk_r.push_back(sinks[k].rate);
    }
    rebuild(*op, (flags & QSW_BUILD_DEFER_NORMS) != 0);
    *out = reinterpret_cast<qsw_op*>(op.release());
  });
}

qsw_status qsw_build_gqsw(qsw_ctx* ctx, const qsw_csr* G, const qsw_csr* H, double omega,
                          const qsw_port* sources, int32_t n_sources, const qsw_port* sinks,
                          int32_t n_sinks, int32_t precision, qsw_op** out) {
  return guarded(ctx, [&] {
    QSW_CHECK_ARG(ctx != nullptr && out != nullptr, QSW_ERR_INVALID_ARG, "ctx/out is NULL");
    check_csr(G, "G", false);
    for (int e = 0; e < G->nnz; ++e)
      QSW_CHECK_ARG(G->w[e] > 0.0, QSW_ERR_NOT_SIMPLE, "G: arc weights must be > 0");
    qsw::ZMat h;
    if (H) {
      check_csr(H, "H", true);
      QSW_CHECK_ARG(H->n == G->n, QSW_ERR_INVALID_ARG, "H must be N x N");
      h = zmat_of_real(H);
    } else {
      h = laplacian_undirected(G);
    }
    const qsw::ZMat l = zmat_of_real(G);
    std::vector<double> hre, hi, lre;
    for (auto& v : h.val) hre.push_back(v.real());
    for (auto& v : l.val) lre.push_back(v.real());
    const qsw_zcsr hz{h.n, (int32_t)h.col.size(), h.rowptr.data(), h.col.data(), hre.data(), nullptr};
    const qsw_zcsr lz{l.n, (int32_t)l.col.size(), l.rowptr.data(), l.col.data(), lre.data(), nullptr};
    const qsw_status st = qsw_build_global(ctx, G->n, &hz, &lz, 1, nullptr, omega, sources,
                                           n_sources, sinks, n_sinks, precision, 0, out);
    if (st != QSW_OK) throw Error{st, ctx->last_error};
  });
}

qsw_status qsw_build_nm_gqsw(qsw_ctx* ctx, const qsw_csr* G, double omega, int32_t precision,
                             qsw_op** out) {
  return guarded(ctx, [&] {
    QSW_CHECK_ARG(ctx != nullptr && out != nullptr, QSW_ERR_INVALID_ARG, "ctx/out is NULL");
    check_csr(G, "G", false);
    for (int e = 0; e < G->nnz; ++e)
      QSW_CHECK_ARG(G->w[e] > 0.0, QSW_ERR_NOT_SIMPLE, "G: arc weights must be > 0");
    std::vector<int> off;
    qsw::ZMat hd, ld, hr;
    qsw::nm_construct(G->n, G->rowptr, G->col, G->w, off, hd, ld, hr);
    auto view = [](const qsw::ZMat& m, std::vector<double>& re, std::vector<double>& im) {
      for (auto& v : m.val) {
        re.push_back(v.real());
        im.push_back(v.imag());
      }
      return qsw_zcsr{m.n, (int32_t)m.col.size(), m.rowptr.data(), m.col.data(), re.data(),
                      im.data()};
    };
    std::vector<double> a, b, c, d, e, f;
    const qsw_zcsr hz = view(hd, a, b), lz = view(ld, c, d), rz = view(hr, e, f);
    const qsw_status st = qsw_build_global(ctx, hd.n, &hz, &lz, 1, &rz, omega, nullptr, 0, nullptr,
                                           0, precision, 0, out);
    if (st != QSW_OK) throw Error{st, ctx->last_error};
    Op* op = reinterpret_cast<Op*>(*out);
    op->gq.vset_off = off;
    op->gq.vset_dev.alloc(sizeof(int) * off.size());
    QSW_CUDA_TRY(cudaMemcpyAsync(op->gq.vset_dev.p, off.data(), sizeof(int) * off.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
    QSW_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  });
}

qsw_status qsw_nm_vsets(const qsw_op* h, int32_t* offsets) {
  const Op* op = reinterpret_cast<const Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op && offsets, QSW_ERR_INVALID_ARG, "op/offsets is NULL");
    QSW_CHECK_ARG(!op->gq.vset_off.empty(), QSW_ERR_INVALID_ARG, "not an NM-G-QSW operator");
    memcpy(offsets, op->gq.vset_off.data(), sizeof(int32_t) * op->gq.vset_off.size());
  });
}

qsw_status qsw_nm_populations(const qsw_op* h, const double* d_pops_expanded, int32_t count,
                              double* d_pops) {
  const Op* op = reinterpret_cast<const Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op && d_pops_expanded && d_pops && count >= 0, QSW_ERR_INVALID_ARG,
                  "bad arguments to qsw_nm_populations");
    QSW_CHECK_ARG(!op->gq.vset_off.empty(), QSW_ERR_INVALID_ARG, "not an NM-G-QSW operator");
    set_device(op->ctx);
    if (count) qsw::nm_populations(*op, d_pops_expanded, count, d_pops);
    QSW_CUDA_TRY(cudaStreamSynchronize(op->ctx->stream));
  });
}

qsw_status qsw_nm_initial_state(const qsw_op* h, const double* h_pops, double* d_state) {
  const Op* op = reinterpret_cast<const Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op && h_pops && d_state, QSW_ERR_INVALID_ARG, "op/pops/d_state is NULL");
    QSW_CHECK_ARG(!op->gq.vset_off.empty(), QSW_ERR_INVALID_ARG, "not an NM-G-QSW operator");
    const int N = (int)op->gq.vset_off.size() - 1;
    double sum = 0.0;
    for (int v = 0; v < N; ++v) {
      QSW_CHECK_ARG(isfinite(h_pops[v]) && h_pops[v] >= 0.0, QSW_ERR_INVALID_ARG,
                    "populations must be finite and >= 0");
      sum += h_pops[v];
    }
    QSW_CHECK_ARG(fabs(sum - 1.0) <= 1e-12, QSW_ERR_INVALID_ARG, "populations must sum to 1");
    set_device(op->ctx);
    qsw::DevBuf p;
    p.alloc(sizeof(double) * N);
    QSW_CUDA_TRY(cudaMemcpyAsync(p.p, h_pops, sizeof(double) * N, cudaMemcpyHostToDevice,
                                 op->ctx->stream));
    qsw::nm_initial_state(*op, p.as<double>(), d_state);
    QSW_CUDA_TRY(cudaStreamSynchronize(op->ctx->stream));
  });
}

qsw_status qsw_set_omega(qsw_op* h, double omega) {
  Op* op = reinterpret_cast<Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op != nullptr, QSW_ERR_INVALID_ARG, "op is NULL");
    QSW_CHECK_ARG(isfinite(omega) && omega >= 0.0 && omega <= 1.0, QSW_ERR_OMEGA_RANGE,
                  "omega must lie in [0, 1]");
    set_device(op->ctx);
    op->omega = omega;
    rebuild(*op, !op->norms_ready);
  });
}

qsw_status qsw_op_info(const qsw_op* h, int64_t* n_tilde, int64_t* n, int64_t* nnz,
                       double* norms9) {
  const Op* op = reinterpret_cast<const Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op != nullptr, QSW_ERR_INVALID_ARG, "op is NULL");
    if (n_tilde) *n_tilde = op->Nt;
    if (n) *n = op->n;
    if (nnz) *nnz = op->nnz_csr;
    if (norms9) {
      ensure_norms(*const_cast<Op*>(op));
      memcpy(norms9, op->norms, sizeof(double) * qsw::kNormPowers);
    }
  });
}

qsw_status qsw_op_export_csr(const qsw_op* h, int32_t* d_rowptr, int32_t* d_col, double* d_val) {
  const Op* op = reinterpret_cast<const Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op != nullptr, QSW_ERR_INVALID_ARG, "op is NULL");
    set_device(op->ctx);
    cudaStream_t st = op->ctx->stream;
    QSW_CHECK_ARG(!op->gq.active, QSW_ERR_INVALID_ARG,
                  "global-interaction walks are matrix-free only (no CSR form)");
    qsw::Csr tmp;
    const qsw::Csr* L = &op->L;
    if (op->opkind != QSW_OPERATOR_CSR) {   // assemble on demand, FP64
      qsw::assemble(*const_cast<Op*>(op), false, tmp);
      L = &tmp;
    }
    if (d_rowptr)
      QSW_CUDA_TRY(cudaMemcpyAsync(d_rowptr, L->rowptr.p, sizeof(int) * (op->n + 1),
                                   cudaMemcpyDeviceToDevice, st));
    if (d_col)
      QSW_CUDA_TRY(cudaMemcpyAsync(d_col, L->col.p, sizeof(int) * L->nnz,
                                   cudaMemcpyDeviceToDevice, st));
    if (d_val) {
      if (!L->fp32) {
        QSW_CUDA_TRY(cudaMemcpyAsync(d_val, L->val.p, sizeof(double2) * L->nnz,
                                     cudaMemcpyDeviceToDevice, st));
      } else {
        qsw::widen_values(*op, d_val);
      }
    }
    QSW_CUDA_TRY(cudaStreamSynchronize(st));
  });
}

void qsw_op_destroy(qsw_op* h) {
  Op* op = reinterpret_cast<Op*>(h);
  if (!op) return;
  cudaSetDevice(op->ctx->device);
  qsw::current_stream() = op->ctx->stream;
  delete op;   // buffers are released in stream order after the op's pending work
}

qsw_status qsw_initial_state(const qsw_op* h, const double* h_rho0, const double* h_pops,
                             double* d_state) {
  const Op* op = reinterpret_cast<const Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op != nullptr && d_state != nullptr, QSW_ERR_INVALID_ARG, "op/d_state is NULL");
    QSW_CHECK_ARG((h_rho0 != nullptr) != (h_pops != nullptr), QSW_ERR_INVALID_ARG,
                  "give exactly one of rho0 and populations");
    set_device(op->ctx);
    cudaStream_t st = op->ctx->stream;
    const int Nt = op->Nt;
    double tr = 0.0;
    if (h_pops) {
      for (int i = 0; i < Nt; ++i) {
        QSW_CHECK_ARG(isfinite(h_pops[i]) && h_pops[i] >= 0.0, QSW_ERR_INVALID_ARG,
                      "populations must be finite and >= 0");
        tr += h_pops[i];
      }
      QSW_CHECK_ARG(fabs(tr - 1.0) <= 1e-12, QSW_ERR_INVALID_ARG, "populations must sum to 1");
      qsw::DevBuf tmp;
      tmp.alloc(sizeof(double) * Nt);
      QSW_CUDA_TRY(cudaMemcpyAsync(tmp.p, h_pops, sizeof(double) * Nt, cudaMemcpyHostToDevice, st));
      qsw::initial_state_from_pops(*op, tmp.as<double>(), d_state);
      QSW_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      for (int i = 0; i < Nt; ++i) tr += h_rho0[2 * ((size_t)i * Nt + i)];
      QSW_CHECK_ARG(fabs(tr - 1.0) <= 1e-12, QSW_ERR_INVALID_ARG, "Tr rho0 must be 1");
      QSW_CUDA_TRY(cudaMemcpyAsync(d_state, h_rho0, sizeof(double2) * op->n, cudaMemcpyHostToDevice,
                                   st));
      QSW_CUDA_TRY(cudaStreamSynchronize(st));
    }
  });
}

qsw_status qsw_apply(const qsw_op* h, const double* d_x, double* d_y) {
  const Op* op = reinterpret_cast<const Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op != nullptr && d_x && d_y && d_x != d_y, QSW_ERR_INVALID_ARG,
                  "bad arguments to qsw_apply");
    set_device(op->ctx);
    qsw::apply(*op, d_x, d_y);
  });
}

static void check_series_args(const Op* op, const void* rho0, double t0, double dt, int steps,
                              const void* out, const void* pops) {
  QSW_CHECK_ARG(op != nullptr && rho0 != nullptr, QSW_ERR_INVALID_ARG, "op/rho0 is NULL");
  QSW_CHECK_ARG(out != nullptr || pops != nullptr, QSW_ERR_INVALID_ARG,
                "give an output array and/or a populations array");
  QSW_CHECK_ARG(steps >= 0, QSW_ERR_INVALID_ARG, "steps must be >= 0");
  QSW_CHECK_ARG(isfinite(t0) && t0 >= 0.0 && isfinite(dt) && dt >= 0.0, QSW_ERR_INVALID_ARG,
                "t0 and dt must be finite and >= 0");
  QSW_CHECK_ARG(isfinite(t0 + steps * dt), QSW_ERR_INVALID_ARG, "time grid overflows");
}

qsw_status qsw_expmv_series(qsw_op* h, const double* d_rho0, double t0, double dt, int32_t steps,
                            double* d_out, double* d_pops, qsw_series_stats* stats) {
  Op* op = reinterpret_cast<Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    check_series_args(op, d_rho0, t0, dt, steps, d_out, d_pops);
    set_device(op->ctx);
    ensure_norms(*op);
    qsw::run_series(*op, d_rho0, t0, dt, steps, d_out, d_pops, stats);
  });
}

qsw_status qsw_expmv_series_noalloc(qsw_op* h, const double* d_rho0, double t0, double dt,
                                    int32_t steps, double* d_out, double* d_pops,
                                    qsw_series_stats* stats) {
  Op* op = reinterpret_cast<Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    check_series_args(op, d_rho0, t0, dt, steps, d_out, d_pops);
    QSW_CHECK_ARG(op->norms_ready, QSW_ERR_INVALID_ARG,
                  "operator built with QSW_BUILD_DEFER_NORMS: its norms need workspace; "
                  "run qsw_expmv_series once first");
    QSW_CHECK_ARG(!op->gq.active, QSW_ERR_INVALID_ARG,
                  "global-interaction walks need a pass-A workspace; use qsw_expmv_series");
    set_device(op->ctx);
    qsw::run_series_noalloc(*op, d_rho0, t0, dt, steps, d_out, d_pops, stats);
  });
}

qsw_status qsw_expmv_series_host(qsw_op* h, const double* h_rho0, double t0, double dt,
                                 int32_t steps, double* h_out, double* h_pops,
                                 qsw_series_stats* stats) {
  Op* op = reinterpret_cast<Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    check_series_args(op, h_rho0, t0, dt, steps, h_out, h_pops);
    set_device(op->ctx);
    ensure_norms(*op);
    cudaStream_t st = op->ctx->stream;
    qsw::DevBuf rho0, out, pops;
    rho0.alloc(sizeof(double2) * op->n);
    if (h_out) out.alloc(sizeof(double2) * op->n * ((size_t)steps + 1));
    if (h_pops) pops.alloc(sizeof(double) * op->Nt * ((size_t)steps + 1));
    QSW_CUDA_TRY(cudaMemcpyAsync(rho0.p, h_rho0, sizeof(double2) * op->n, cudaMemcpyHostToDevice, st));
    if (h_out) {
      // outputs are copied to the host on a second stream as the series kernel
      // finishes them, overlapping the copies with the remaining Taylor blocks
      qsw_ctx* c = op->ctx;
      if (!c->copy) QSW_CUDA_TRY(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking));
      if (!c->count_h) {
        QSW_CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&c->count_h), sizeof(int),
                                   cudaHostAllocMapped));
        QSW_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->count_d), c->count_h, 0));
      }
      *(volatile int*)c->count_h = 0;
      const size_t vb = sizeof(double2) * (size_t)op->n;
      int copied = 0;
      struct Drain {   // the copy stream must be idle before `out` is released
        cudaStream_t s;
        ~Drain() { cudaStreamSynchronize(s); }
      } drain{c->copy};
      qsw::OutputSink sink{c->count_h, c->count_d, [&](int k) {
        QSW_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(h_out) + vb * copied,
                                     static_cast<char*>(out.p) + vb * copied, vb * (k - copied),
                                     cudaMemcpyDeviceToHost, c->copy));
        copied = k;
      }};
      qsw::run_series(*op, rho0.as<double>(), t0, dt, steps, out.as<double>(),
                      h_pops ? pops.as<double>() : nullptr, stats, &sink);
      if (copied < steps + 1)
        QSW_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(h_out) + vb * copied,
                                     static_cast<char*>(out.p) + vb * copied,
                                     vb * (steps + 1 - copied), cudaMemcpyDeviceToHost, st));
      QSW_CUDA_TRY(cudaStreamSynchronize(c->copy));
    } else {
      qsw::run_series(*op, rho0.as<double>(), t0, dt, steps, nullptr,
                      h_pops ? pops.as<double>() : nullptr, stats);
    }
    if (h_pops)
      QSW_CUDA_TRY(cudaMemcpyAsync(h_pops, pops.p, sizeof(double) * op->Nt * ((size_t)steps + 1),
                                   cudaMemcpyDeviceToHost, st));
    QSW_CUDA_TRY(cudaStreamSynchronize(st));
  });
}

qsw_status qsw_populations(const qsw_op* h, const double* d_rho, int32_t count, double* d_pops) {
  const Op* op = reinterpret_cast<const Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op != nullptr && d_rho && d_pops && count >= 0, QSW_ERR_INVALID_ARG,
                  "bad arguments to qsw_populations");
    if (count == 0) return;
    set_device(op->ctx);
    qsw::populations(*op, d_rho, count, d_pops);
  });
}

int64_t qsw_kernel_launches(void) { return qsw::g_launches.load(); }

int64_t qsw_device_allocations(void) { return qsw::g_device_allocs.load(); }

int64_t qsw_tune_measurements(void) {
  return qsw::tune_measurements() + qsw::batch_tune_measurements();
}

void qsw_tune_reset(void) {
  qsw::tune_reset();
  qsw::batch_tune_reset();
}

qsw_status qsw_batch_set_schedule(qsw_ctx* ctx, int32_t cluster_size, int32_t small_limit) {
  return guarded(ctx, [&] {
    QSW_CHECK_ARG(ctx != nullptr, QSW_ERR_INVALID_ARG, "ctx is NULL");
    QSW_CHECK_ARG(cluster_size == 0 || cluster_size == 2 || cluster_size == 4 ||
                      cluster_size == 8 || cluster_size == 16,
                  QSW_ERR_INVALID_ARG, "cluster_size must be 0, 2, 4, 8 or 16");
    QSW_CHECK_ARG(small_limit >= -1 && small_limit <= 65536, QSW_ERR_INVALID_ARG,
                  "small_limit must be -1 or 0 .. 65536");
    ctx->batch_cs = cluster_size;
    ctx->batch_small = small_limit;
  });
}

qsw_status qsw_op_set_csr_schedule(qsw_op* h, int32_t csr_lanes_per_row, int32_t csr_unroll) {
  Op* op = reinterpret_cast<Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op != nullptr && op->opkind == QSW_OPERATOR_CSR, QSW_ERR_INVALID_ARG,
                  "a CSR operator is required");
    const int l = csr_lanes_per_row;
    QSW_CHECK_ARG(l == -1 || l == 1 || l == 2 || l == 4 || l == 8 || l == 16 || l == 32,
                  QSW_ERR_INVALID_ARG, "csr_lanes_per_row must be -1, 1, 2, 4, 8, 16 or 32");
    QSW_CHECK_ARG(csr_unroll == 2 || csr_unroll == 4, QSW_ERR_INVALID_ARG, "csr_unroll must be 2 or 4");
    op->tpr_fixed = true;
    op->csr_sell = l < 0;
    if (l > 0) {
      op->tpr = l;
      op->sell = qsw::Sell{};
    }
    op->csr_unroll = csr_unroll;
  });
}

qsw_status qsw_op_schedule(const qsw_op* op, int32_t* csr_lanes_per_row, int32_t* csr_unroll) {
  if (!op || !csr_lanes_per_row) return QSW_ERR_INVALID_ARG;
  const Op* o = reinterpret_cast<const Op*>(op);
  const bool csr = o->opkind == QSW_OPERATOR_CSR;
  *csr_lanes_per_row = csr ? (o->csr_sell ? -1 : o->tpr) : 0;
  if (csr_unroll) *csr_unroll = csr ? o->csr_unroll : 0;
  return QSW_OK;
}

qsw_status qsw_batch_series(qsw_ctx* ctx, int32_t count, qsw_op* const* ops,
                            const double* const* d_rho0, int32_t n0, const double* t0,
                            const double* dt, const int32_t* steps, double* const* d_pops,
                            qsw_batch_stats* stats) {
  return guarded(ctx, [&] {
    QSW_CHECK_ARG(ctx && count >= 1 && ops && d_rho0 && t0 && dt && steps && d_pops,
                  QSW_ERR_INVALID_ARG, "bad arguments to qsw_batch_series");
    for (int w = 0; w < count; ++w) {
      QSW_CHECK_ARG(ops[w] && d_rho0[w] && d_pops[w], QSW_ERR_INVALID_ARG, "NULL walk pointer");
      QSW_CHECK_ARG(reinterpret_cast<Op*>(ops[w])->ctx == ctx, QSW_ERR_INVALID_ARG,
                    "operator from another context");
      check_series_args(reinterpret_cast<Op*>(ops[w]), d_rho0[w], t0[w], dt[w], steps[w], nullptr,
                        d_pops[w]);
    }
    set_device(ctx);
    qsw::run_batch(ctx, count, reinterpret_cast<Op* const*>(ops), d_rho0, n0, t0, dt, steps,
                   d_pops, stats);
  });
}

qsw_status qsw_survival_time(qsw_op* h, const double* d_rho0, double t_end, int32_t q,
                             int32_t sink, double* eta, double* d_pops, qsw_series_stats* stats) {
  Op* op = reinterpret_cast<Op*>(h);
  return guarded(op ? op->ctx : nullptr, [&] {
    QSW_CHECK_ARG(op && d_rho0 && eta, QSW_ERR_INVALID_ARG, "op/rho0/eta is NULL");
    set_device(op->ctx);
    ensure_norms(*op);
    qsw::run_survival(*op, d_rho0, t_end, q, sink, eta, d_pops, stats);
  });
}

qsw_status qsw_batch_survival_time(qsw_ctx* ctx, int32_t count, qsw_op* const* ops,
                                   const double* const* d_rho0, const double* t_end,
                                   const int32_t* q, const int32_t* sink, double* eta,
                                   qsw_batch_stats* stats) {
  return guarded(ctx, [&] {
    QSW_CHECK_ARG(ctx && count >= 1 && ops && d_rho0 && t_end && q && sink && eta,
                  QSW_ERR_INVALID_ARG, "bad arguments to qsw_batch_survival_time");
    for (int w = 0; w < count; ++w) {
      QSW_CHECK_ARG(ops[w] && d_rho0[w], QSW_ERR_INVALID_ARG, "NULL walk pointer");
      QSW_CHECK_ARG(reinterpret_cast<Op*>(ops[w])->ctx == ctx, QSW_ERR_INVALID_ARG,
                    "operator from another context");
    }
    set_device(ctx);
    qsw::run_batch_survival(ctx, count, reinterpret_cast<Op* const*>(ops), d_rho0, t_end, q, sink,
                            eta, stats);
  });
}

qsw_status qsw_probe_wait_limit(qsw_ctx* ctx, double* seconds) {
  return guarded(ctx, [&] {
    QSW_CHECK_ARG(ctx != nullptr, QSW_ERR_INVALID_ARG, "ctx is NULL");
    set_device(ctx);
    const double s = qsw::probe_wait_limit(ctx);
    if (seconds) *seconds = s;
  });
}

qsw_status qsw_theta_table(int32_t precision, double* theta55) {
  return guarded(nullptr, [&] {
    QSW_CHECK_ARG(theta55 != nullptr, QSW_ERR_INVALID_ARG, "theta55 is NULL");
    QSW_CHECK_ARG(precision == QSW_C128 || precision == QSW_C64_BULK, QSW_ERR_INVALID_ARG,
                  "unknown precision");
    memcpy(theta55, qsw::theta_table(precision), sizeof(double) * qsw::kMMax);
  });
}

qsw_status qsw_select_params(const double* norms9, double t, int32_t n0, int32_t precision,
                             int32_t* m_star, int32_t* s) {
  return guarded(nullptr, [&] {
    QSW_CHECK_ARG(norms9 && m_star && s, QSW_ERR_INVALID_ARG, "NULL argument");
    QSW_CHECK_ARG(n0 >= 1 && isfinite(t) && t >= 0.0, QSW_ERR_INVALID_ARG, "bad t or n0");
    QSW_CHECK_ARG(precision == QSW_C128 || precision == QSW_C64_BULK, QSW_ERR_INVALID_ARG,
                  "unknown precision");
    double dp[qsw::kNormPowers + 1] = {0};
    dp[0] = norms9[0];
    for (int p = 2; p <= qsw::kNormPowers; ++p) dp[p - 1] = pow(norms9[p - 1], 1.0 / p);
    const qsw::Params r = qsw::select_params(dp, qsw::theta_table(precision), t, n0);
    *m_star = r.m;
    *s = r.s;
  });
}

}  // extern "C"
