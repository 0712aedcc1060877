// Al-Mohy & Higham parameter choice (Code Fragment 3.1) and the series plan
// (Algorithms 3.2 / 5.2) as one piece of code compiled for host and device.
//
// Only IEEE-exact operations (+, *, /, ceil, comparisons) appear here, so the
// host copy (used to size the workspace) and the device copy (which decides
// what the series kernel runs) agree bit for bit on the same inputs.
#pragma once

#include <math.h>

#include "qsw_internal.h"

namespace qsw {

// A-H eq. (3.13): ||tA||_1 small enough that p = 1 alone decides.
__host__ __device__ inline bool small_norm_condition(double norm1, const double* theta, int n0) {
  return norm1 <= 2 * kEll * kPMax * (kPMax + 3) * theta[kMMax - 1] / (n0 * kMMax);
}

__host__ __device__ inline Params select_params(const double* dp, const double* theta, double t,
                                                int n0) {
  Params out{0, 1};
  const double norm1 = t * dp[0];
  if (!(norm1 > 0.0)) return out;   // t ||A||_1 = 0: exp(tA)b = b
  double best_cost = -1.0;
  int best_m = 0;
  if (small_norm_condition(norm1, theta, n0)) {
    for (int m = 1; m <= kMMax; ++m) {
      const double cost = m * ceil(norm1 / theta[m - 1]);
      if (best_cost < 0.0 || cost < best_cost) {
        best_cost = cost;
        best_m = m;
      }
    }
    out.m = best_m;
    out.s = (int)(best_cost / best_m);
    return out;
  }
  for (int m = 1; m <= kMMax; ++m) {
    double cm = -1.0;   // C_m = min over admissible p of m * ceil(alpha_p / theta_m)
    for (int p = 2; p <= kPMax; ++p) {
      if (p * (p - 1) - 1 > m) break;
      const double alpha = dp[p - 1] > dp[p] ? dp[p - 1] : dp[p];
      const double c = m * ceil(t * alpha / theta[m - 1]);
      if (cm < 0.0 || c < cm) cm = c;
    }
    if (best_cost < 0.0 || cm < best_cost) {
      best_cost = cm;
      best_m = m;
    }
  }
  out.m = best_m;
  const double s = best_cost / best_m;
  out.s = s < 1.0 ? 1 : (int)s;
  return out;
}

// Series plan.  Series index k (state at t0 + k dt) lives in slot
// (ring ? k % ring : k).  Job.z_slot / out slots are series indices here; the
// kernel maps them to memory with the same rule.
__host__ __device__ inline PlanInfo plan_series(const double* dp, const double* theta, double t0,
                                                double dt, int steps, int n0, int ring, Job* jobs,
                                                int max_jobs, int dmax) {
  PlanInfo info{};
  int nj = 0;
  // one block of d outputs sharing Z, as ceil(d / dmax) jobs
  auto push = [&](int z, int out0, int d, int m, int fin, double hspan) {
    if (d > info.max_d) info.max_d = d;
    for (int k0 = 0; k0 < d; k0 += dmax) {
      const int dc = d - k0 < dmax ? d - k0 : dmax;
      if (jobs && nj < max_jobs) {
        Job& j = jobs[nj];
        j.z_slot = z;
        j.out_slot0 = out0 + k0;
        j.out_index0 = out0 + k0;
        j.d = dc;
        j.m = m;
        j.final_outputs = fin;
        j.k_off = k0;
        j.d_block = d;
        j.hspan = hspan;
      }
      ++nj;
      info.outputs += dc;
      if (dc > info.max_job_d) info.max_job_d = dc;
    }
  };
  (void)ring;
  // State 0: Algorithm 3.2 for t0 A with its own parameters; stage i feeds
  // stage i + 1 through the same slot.
  const Params p0 = select_params(dp, theta, t0, n0);
  info.m0 = p0.m;
  info.s0 = p0.s;
  for (int i = 0; i < p0.s; ++i)
    push(i == 0 ? -1 : 0, 0, 1, p0.m, i == p0.s - 1, p0.m ? t0 / p0.s : 0.0);
  if (steps > 0) {
    const Params ps = select_params(dp, theta, steps * dt, n0);
    info.m_star = ps.m;
    info.s = ps.s;
    if (steps <= ps.s) {
      // Algorithm 5.2 with q <= s: each dt step by Algorithm 3.2.
      const Params ph = select_params(dp, theta, dt, n0);
      info.step_m = ph.m;
      info.step_s = ph.s;
      for (int k = 0; k < steps; ++k)
        for (int i = 0; i < ph.s; ++i)
          push(i == 0 ? k : k + 1, k + 1, 1, ph.m, i == ph.s - 1, ph.m ? dt / ph.s : 0.0);
    } else {
      // Algorithm 5.2: j blocks of d outputs reusing Taylor powers, plus a
      // remainder block of r outputs.
      const int d = steps / ps.s;
      const int jb = steps / d;
      const int r = steps - d * jb;
      info.d = d;
      for (int i = 1; i <= jb + 1; ++i) {
        const int dd = i <= jb ? d : r;
        if (dd == 0) break;
        push((i - 1) * d, (i - 1) * d + 1, dd, ps.m, 1, dd * dt);
      }
    }
  }
  info.njobs = nj;
  return info;
}

}  // namespace qsw
