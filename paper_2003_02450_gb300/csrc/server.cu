// Serving runtime: a request loop for L-QSW time series (not in the paper).
//
// Requests (a graph, omega, rho0, a time grid, a precision) arrive from any
// host thread.  W worker threads each own a CUDA stream and a library context.
// A free worker takes every queued request that fits the device-memory budget
// (first come, first served, up to max_batch), builds their superoperators on
// its stream, uploads their initial states, and runs them as ONE batched launch
// (batch.cu: a thread-block cluster per walk).  A walk's cluster raises a
// host-mapped flag when the walk's populations are final; the worker polls the
// flags while the launch runs, copies each finished walk's populations to the
// caller on its copy stream and completes that request at once, so a short
// walk does not wait for the longest walk of its batch.  While one worker's
// batch is on the GPU, requests that arrive are taken by another worker and
// launched on its stream, so their work overlaps on the device (continuous
// batching at launch granularity, completion at walk granularity).  A batch's
// device memory is released in stream order when its launch ends (and only then
// counted free for admission), so no worker ever synchronises the whole device.
//
// Workers take the batched series phase's schedule from the tuner's cache
// (filled by earlier qsw_batch_series calls) and never time candidates
// themselves, so no request waits for a tuning pass.
//
// A walk's result does not depend on the other walks of its batch: each walk
// is computed by its own cluster with its own reductions in a fixed order, so a
// request gives the same populations alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <string.h>

#include "op.h"

struct qsw_server;

namespace qsw {
namespace {

using Clock = std::chrono::steady_clock;

// Requests with at least this many vertices (n = N^2 >= 25,600 elements) run
// on the whole GPU; a cluster of 8 CTAs is ~3 % of the machine.
constexpr int kWholeGpuVertices = 160;

struct Req {
  int64_t id = 0;
  // inputs (host copies)
  int N = 0;
  std::vector<int> rowptr, col;
  std::vector<double> w;
  double omega = 0.0;
  int precision = QSW_C128;
  std::vector<double> rho0;   // 2 n doubles (complex128) or empty
  std::vector<double> pops0;  // N~ doubles or empty
  double t0 = 0.0, dt = 0.0;
  int steps = 0;
  double* pops_out = nullptr; // caller's host buffer
  size_t footprint = 0;
  // outcome
  int done = 0;
  qsw_status status = QSW_OK;
  std::string error;
  Clock::time_point t_submit, t_start, t_done;
  int64_t matvecs = 0;
};

size_t footprint_of(int N, int steps, int precision) {
  // upper bound of device memory a request holds while it runs: operator data,
  // the initial state, populations, the norm workspace (6 vectors + h), two
  // Taylor terms and a ring of at most steps + 1 FP64 accumulators
  const double n = (double)N * N;
  const double vb = precision == QSW_C64_BULK ? 8.0 : 16.0;
  const double bytes = n * (16.0 + 104.0 + 2.0 * vb + 16.0 * (steps + 2)) +
                       (double)(steps + 1) * N * 8.0 + 64.0 * N + (1 << 20);
  return (size_t)bytes;
}

}  // namespace
}  // namespace qsw

struct qsw_server {
  int device = 0;
  int workers = 2;
  int max_batch = 64;
  size_t budget = 0;
  size_t in_use = 0;
  bool stopping = false;
  int64_t next_id = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<qsw::Req>> queue;
  std::map<int64_t, std::shared_ptr<qsw::Req>> all;
  std::vector<std::thread> threads;
  std::vector<qsw_ctx*> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaStream_t> copy_streams;  // per worker: early copies of finished walks
  std::vector<int*> done_h;                // per worker: host-mapped completion flags
  std::vector<int*> done_d;                //   (max_batch each) and their device addresses
  int64_t batches = 0;
  int64_t early = 0;                       // requests completed before their batch ended

  void complete(const std::shared_ptr<qsw::Req>& r, qsw::Clock::time_point t);

  void worker(int wi);
};

// Marks one request done (its populations are on the host) and wakes waiters.
void qsw_server::complete(const std::shared_ptr<qsw::Req>& r, qsw::Clock::time_point t) {
  {
    std::lock_guard<std::mutex> lk(mu);
    if (r->done) return;
    r->t_done = t;
    r->done = 1;
  }
  cv_done.notify_all();
}

void qsw_server::worker(int wi) {
  using namespace qsw;
  cudaSetDevice(device);
  qsw_ctx* ctx = ctxs[wi];
  current_stream() = ctx->stream;
  for (;;) {
    std::vector<std::shared_ptr<Req>> take;
    {
      std::unique_lock<std::mutex> lk(mu);
      // wake for shutdown, or when the oldest request fits the budget (or the
      // device holds nothing, so that an oversized request still runs alone)
      cv_work.wait(lk, [&] {
        return stopping ||
               (!queue.empty() && (in_use == 0 || in_use + queue.front()->footprint <= budget));
      });
      if (queue.empty() && stopping) return;
      if (queue.empty()) continue;
      // first come, first served, as long as the memory budget allows; the
      // head of the queue is always taken when nothing else runs.  A large
      // walk (whole-GPU kernel) is taken alone; small walks are grouped into
      // one batched launch and never wait behind a large one.
      if (queue.front()->N >= kWholeGpuVertices) {
        auto r = queue.front();
        in_use += r->footprint;
        take.push_back(r);
        queue.pop_front();
      } else {
        for (auto it = queue.begin(); it != queue.end() && (int)take.size() < max_batch;) {
          auto& r = *it;
          if (r->N >= kWholeGpuVertices) { ++it; continue; }
          if (in_use + r->footprint > budget && !(in_use == 0 && take.empty())) break;
          in_use += r->footprint;
          take.push_back(r);
          it = queue.erase(it);
        }
      }
      if (!take.empty()) ++batches;
    }
    if (take.empty()) continue;
    const auto t_start = Clock::now();
    for (auto& r : take) r->t_start = t_start;
    // build operators and upload inputs on this worker's stream
    std::vector<qsw_op*> ops;
    std::vector<std::shared_ptr<Req>> live;
    std::vector<DevBuf> rho(take.size()), pops(take.size());
    std::vector<const double*> d_rho;
    std::vector<double*> d_pops;
    std::vector<double> t0s, dts;
    std::vector<int> steps;
    std::vector<double*> pinned;
    for (size_t k = 0; k < take.size(); ++k) {
      Req& r = *take[k];
      qsw_csr g{r.N, (int32_t)r.col.size(), r.rowptr.data(), r.col.data(), r.w.data()};
      qsw_op* op = nullptr;
      qsw_status st = qsw_build_superoperator(ctx, &g, nullptr, r.omega, nullptr, 0, nullptr, 0,
                                              r.precision,
                                              QSW_OPERATOR_MATRIX_FREE | QSW_BUILD_DEFER_NORMS, &op);
      if (st == QSW_OK) {
        const long long n = (long long)r.N * r.N;
        try {
          rho[k].alloc(sizeof(double2) * n);
          pops[k].alloc(sizeof(double) * (size_t)(r.steps + 1) * r.N);
          if (!r.rho0.empty())
            st = cudaMemcpyAsync(rho[k].p, r.rho0.data(), sizeof(double2) * n,
                                 cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess
                     ? QSW_OK
                     : QSW_ERR_CUDA;
          else
            st = qsw_initial_state(op, nullptr, r.pops0.data(), rho[k].as<double>());
        } catch (const Error& e) {
          st = e.status;
        }
      }
      if (st != QSW_OK) {
        r.status = st;
        r.error = ctx->last_error;
        if (op) qsw_op_destroy(op);
        continue;
      }
      ops.push_back(op);
      live.push_back(take[k]);
      d_rho.push_back(rho[k].as<double>());
      d_pops.push_back(pops[k].as<double>());
      t0s.push_back(r.t0);
      dts.push_back(r.dt);
      steps.push_back(r.steps);
    }
    qsw_status st = QSW_OK;
    std::string err;
    if (!ops.empty()) {
      // large walks use the whole GPU (the persistent single-walk kernel); the
      // rest share one batched launch, a thread-block cluster each
      std::vector<qsw_op*> bops;
      std::vector<const double*> brho;
      std::vector<double*> bpops;
      std::vector<double> bt0, bdt;
      std::vector<int> bsteps;
      for (size_t k = 0; k < live.size(); ++k) {
        Req& r = *live[k];
        if (r.N >= kWholeGpuVertices) {
          const qsw_status s1 = qsw_expmv_series(ops[k], d_rho[k], r.t0, r.dt, r.steps, nullptr,
                                                 d_pops[k], nullptr);
          if (s1 != QSW_OK) {
            r.status = s1;
            r.error = ctx->last_error;
          }
          continue;
        }
        bops.push_back(ops[k]);
        brho.push_back(d_rho[k]);
        bpops.push_back(d_pops[k]);
        bt0.push_back(t0s[k]);
        bdt.push_back(dts[k]);
        bsteps.push_back(steps[k]);
      }
      if (!bops.empty()) {
        // one batched launch; each walk's populations go to its caller as soon
        // as its cluster (or CTA) has finished it, while the others still run
        std::vector<std::shared_ptr<Req>> breqs;
        for (size_t k = 0; k < live.size(); ++k)
          if (live[k]->N < kWholeGpuVertices) breqs.push_back(live[k]);
        for (size_t w = 0; w < bops.size(); ++w) done_h[wi][w] = 0;
        cudaStream_t cs = copy_streams[wi];
        WalkSink sink{done_h[wi], done_d[wi], [&](int w) {
                        Req& r = *breqs[w];
                        if (r.status != QSW_OK) return;
                        if (cudaMemcpyAsync(r.pops_out, bpops[w],
                                            sizeof(double) * (size_t)(r.steps + 1) * r.N,
                                            cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
                            cudaStreamSynchronize(cs) != cudaSuccess)
                          return;   // left to the copy after the launch
                        complete(breqs[w], Clock::now());
                        std::lock_guard<std::mutex> lk(mu);
                        ++early;
                      }};
        try {
          for (qsw_op* op : bops)
            QSW_CHECK_ARG(reinterpret_cast<Op*>(op)->ctx == ctx, QSW_ERR_INVALID_ARG,
                          "operator from another context");
          qsw::run_batch(ctx, (int)bops.size(), reinterpret_cast<Op* const*>(bops.data()),
                         brho.data(), 1, bt0.data(), bdt.data(), bsteps.data(), bpops.data(),
                         nullptr, &sink);
        } catch (const Error& e) {
          st = e.status;
          err = e.msg;
        }
      }
      if (st != QSW_OK && err.empty()) err = ctx->last_error;
      for (size_t k = 0; k < live.size() && st == QSW_OK; ++k) {
        Req& r = *live[k];
        if (r.done) continue;   // handed out early
        if (cudaMemcpyAsync(r.pops_out, d_pops[k], sizeof(double) * (size_t)(r.steps + 1) * r.N,
                            cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
          st = QSW_ERR_CUDA;
      }
      if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && st == QSW_OK) st = QSW_ERR_CUDA;
      for (qsw_op* op : ops) qsw_op_destroy(op);
    }
    rho.clear();
    pops.clear();
    const auto t_done = Clock::now();
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto& r : take) {
        if (!r->done) {
          if (r->status == QSW_OK && st != QSW_OK) {
            r->status = st;
            r->error = err;
          }
          r->t_done = t_done;
          r->done = 1;
        }
        in_use -= r->footprint;   // the batch's device memory is released now
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();   // memory freed: queued requests may now fit
  }
}

extern "C" {

qsw_status qsw_server_create(int device, const qsw_server_config* cfg, qsw_server** out) {
  if (!out) return QSW_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<qsw_server> s(new qsw_server());
  s->device = device;
  if (cfg) {
    if (cfg->workers >= 1) s->workers = cfg->workers;
    if (cfg->max_batch >= 1) s->max_batch = cfg->max_batch;
    s->budget = (size_t)cfg->memory_budget_bytes;
  }
  if (cudaSetDevice(device) != cudaSuccess) return QSW_ERR_CUDA;
  if (s->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return QSW_ERR_CUDA;
    s->budget = fr / 2;
  }
  for (int k = 0; k < s->workers; ++k) {
    cudaStream_t st, cs;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return QSW_ERR_CUDA;
    s->streams.push_back(st);
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return QSW_ERR_CUDA;
    s->copy_streams.push_back(cs);
    int* h = nullptr;
    int* d = nullptr;
    if (cudaHostAlloc(reinterpret_cast<void**>(&h), sizeof(int) * s->max_batch, cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&d), h, 0) != cudaSuccess)
      return QSW_ERR_CUDA;
    s->done_h.push_back(h);
    s->done_d.push_back(d);
    qsw_ctx* c = nullptr;
    const qsw_status r = qsw_create(&c, device, st);
    if (r != QSW_OK) return r;
    c->batch_no_tune = true;   // a worker never stalls a batch to time schedules
    s->ctxs.push_back(c);
  }
  for (int k = 0; k < s->workers; ++k) s->threads.emplace_back(&qsw_server::worker, s.get(), k);
  *out = s.release();
  return QSW_OK;
}

qsw_status qsw_server_submit(qsw_server* s, const qsw_request* rq, int64_t* id) {
  if (!s || !rq || !id || !rq->pops_out) return QSW_ERR_INVALID_ARG;
  const qsw_csr& g = rq->graph;
  if (g.n < 1 || !g.rowptr || g.nnz < 0 || (g.nnz > 0 && (!g.col || !g.w))) return QSW_ERR_INVALID_ARG;
  if ((rq->rho0 == nullptr) == (rq->populations == nullptr)) return QSW_ERR_INVALID_ARG;
  if (rq->steps < 0 || !(rq->dt >= 0.0) || !(rq->t0 >= 0.0)) return QSW_ERR_INVALID_ARG;
  if (rq->precision != QSW_C128 && rq->precision != QSW_C64_BULK) return QSW_ERR_INVALID_ARG;
  auto r = std::make_shared<qsw::Req>();
  r->N = g.n;
  r->rowptr.assign(g.rowptr, g.rowptr + g.n + 1);
  r->col.assign(g.col, g.col + g.nnz);
  r->w.assign(g.w, g.w + g.nnz);
  r->omega = rq->omega;
  r->precision = rq->precision;
  const size_t n = (size_t)g.n * g.n;
  if (rq->rho0) r->rho0.assign(rq->rho0, rq->rho0 + 2 * n);
  else r->pops0.assign(rq->populations, rq->populations + g.n);
  r->t0 = rq->t0;
  r->dt = rq->dt;
  r->steps = rq->steps;
  r->pops_out = rq->pops_out;
  r->footprint = qsw::footprint_of(g.n, rq->steps, rq->precision);
  r->t_submit = qsw::Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return QSW_ERR_INVALID_ARG;
    r->id = s->next_id++;
    *id = r->id;
    s->all[r->id] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_one();
  return QSW_OK;
}

qsw_status qsw_server_wait(qsw_server* s, int64_t id, double timeout_s, qsw_request_result* res) {
  if (!s) return QSW_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return QSW_ERR_INVALID_ARG;
  auto r = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&] { return r->done != 0; });
  if (!ok) return QSW_ERR_NOT_CONVERGED;
  if (res) {
    using ms = std::chrono::duration<double, std::milli>;
    res->status = r->status;
    res->latency_ms = ms(r->t_done - r->t_submit).count();
    res->queue_ms = ms(r->t_start - r->t_submit).count();
    strncpy(res->error, r->error.c_str(), sizeof(res->error) - 1);
    res->error[sizeof(res->error) - 1] = 0;
  }
  const qsw_status st = r->status;
  s->all.erase(it);
  return st;
}

qsw_status qsw_server_stats(qsw_server* s, int64_t* queued, int64_t* batches, double* bytes_in_use) {
  if (!s) return QSW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int64_t)s->queue.size();
  if (batches) *batches = s->batches;
  if (bytes_in_use) *bytes_in_use = (double)s->in_use;
  return QSW_OK;
}

void qsw_server_destroy(qsw_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads) t.join();
  for (qsw_ctx* c : s->ctxs) qsw_destroy(c);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (cudaStream_t st : s->copy_streams) cudaStreamDestroy(st);
  for (int* h : s->done_h) cudaFreeHost(h);
  delete s;
}

}  // extern "C"
