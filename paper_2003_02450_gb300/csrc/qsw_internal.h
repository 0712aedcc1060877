// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/qsw.h"

namespace qsw {

constexpr int kMMax = 55;     // m_max of Al-Mohy & Higham Code Fragment 3.1
constexpr int kPMax = 8;      // p_max (largest p with p(p-1) <= m_max + 1)
constexpr int kEll = 2;       // columns of the 1-norm estimator
constexpr int kNormPowers = 9;  // ||L^p||_1, p = 1..9 (paper Section 4 footnote)
constexpr int kMaxPorts = 4096;
constexpr int kMaxGlobalOps = 8;   // Lindblad operators of a global-interaction walk

// Number of kernels this library has launched in this process (all devices).
extern std::atomic<long long> g_launches;
// Number of device allocations (DevBuf::alloc, the library's only device
// allocator) made in this process.
extern std::atomic<long long> g_device_allocs;
#define QSW_LAUNCH ::qsw::g_launches.fetch_add(1, std::memory_order_relaxed),

// ------------------------------------------------------------------ errors
struct Error {
  qsw_status status;
  std::string msg;
};

#define QSW_CUDA_TRY(expr)                                                         \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      throw ::qsw::Error{e_ == cudaErrorMemoryAllocation ? QSW_ERR_OOM : QSW_ERR_CUDA, \
                         std::string(#expr) + ": " + cudaGetErrorString(e_)};      \
    }                                                                              \
  } while (0)

#define QSW_CHECK_ARG(cond, code, text)              \
  do {                                                \
    if (!(cond)) throw ::qsw::Error{(code), (text)};  \
  } while (0)

// ------------------------------------------------------------ device memory
// Stream on which the calling thread's library work runs (set at every API
// entry from the context).  Device buffers are allocated and freed in stream
// order on it (cudaMallocAsync / cudaFreeAsync), so freeing never synchronises
// the whole device and concurrent streams keep running.
inline cudaStream_t& current_stream() {
  static thread_local cudaStream_t s = nullptr;
  return s;
}

// RAII device buffer, stream-ordered on the stream current at allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      s = o.s;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t nbytes) {
    if (nbytes <= bytes && p) return;
    release();
    if (nbytes == 0) return;
    s = current_stream();
    g_device_allocs.fetch_add(1, std::memory_order_relaxed);
    QSW_CUDA_TRY(cudaMallocAsync(&p, nbytes, s));
    bytes = nbytes;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// ----------------------------------------------------- parameter selection
// theta tables (host copy; the device copy lives in __constant__ memory of
// series.cu).  theta[prec][m-1], m = 1..55.
const double* theta_table(int precision);   // computes on first use
double tolerance(int precision);

// Outcome of Code Fragment 3.1 for one matrix t*L.
struct Params {
  int m;
  int s;
};

// dp[0] = ||L||_1 (exact), dp[p-1] = ||L^p||_1^(1/p) for p = 2..9.
// Identical code on host and device (IEEE operations only: *, /, ceil, <=).
__host__ __device__ Params select_params(const double* dp, const double* theta, double t, int n0);

// One Taylor job of the device program: outputs k = k_off + 1 .. k_off + d of
// a block of d_block outputs, F_k = sum_p (k/d_block)^p Khat_p, with
// Khat_p = (hspan/p) L Khat_{p-1}, Khat_0 = Z.  A block with more outputs than
// a kernel keeps state for is split into chunks (k_off > 0 for all but the
// first): every chunk starts again from the block's Z and forms the same
// powers, so each output gets exactly the arithmetic of the unsplit block.
struct Job {
  int z_slot;        // slot of Z (-1: the caller's rho0)
  int out_slot0;     // slot of this job's first output; the rest follow (mod ring)
  int out_index0;    // series index of this job's first output (for populations), or -1
  int d;             // outputs in this job
  int m;             // m* (max Taylor degree)
  int final_outputs; // 1 if the outputs are final series states (write populations)
  int k_off;         // outputs of the block before this job
  int d_block;       // outputs of the whole block (coefficient (k / d_block)^p)
  double hspan;      // d_block * h: Khat_p = (hspan/p) L Khat_{p-1}
};

// Whole-series plan (Algorithm 5.2, with Algorithm 3.2 for the first state
// and for the stepwise branch).  Built identically on host and device.
struct PlanInfo {
  int njobs;
  int max_d;       // largest block (outputs sharing one Z): sizes an output ring
  int max_job_d;   // largest job (<= the chunk limit)
  int outputs;     // sum of the jobs' outputs (each initialised once from its Z)
  int m0, s0, m_star, s, step_m, step_s, d;
};

// Writes up to max_jobs jobs (jobs may be null to only count).  `ring` > 0
// maps series index k to slot k % ring (workspace ring); ring == 0 maps index
// k to slot k (caller's output array).  Blocks of more than `dmax` outputs are
// split into ceil(d / dmax) jobs.
__host__ __device__ PlanInfo plan_series(const double* dp, const double* theta, double t0,
                                         double dt, int steps, int n0, int ring, Job* jobs,
                                         int max_jobs, int dmax);

}  // namespace qsw
