// Per-step coefficients of the Adam-family optimisers (rules in fpm.h), computed
// on the host in FP64 and handed to the update kernel as four floats per step.
// Host-only and free of CUDA calls, so the CPU tests compile it with g++.
#pragma once

#include <cmath>

#include "../../include/fpm.h"

namespace fpmk {

// NAdam's momentum coefficient of step t: b1 (1 - 0.96^(0.004 t) / 2).
inline double nadam_mu(double b1, double t) { return b1 * (1.0 - 0.5 * std::pow(0.96, 0.004 * t)); }

// The running product P_t = mu_1 ... mu_t, advanced from (t0, p0) to t.
inline double nadam_advance(double b1, long long t0, double p0, long long t) {
  for (long long k = t0 + 1; k <= t; ++k) p0 *= nadam_mu(b1, (double)k);
  return p0;
}

// Coefficients of step t (>= 1) for optimiser opt, given P_(t-1) for NAdam:
//   Adam, AdamW: (1/(1-b1^t), 1/sqrt(1-b2^t), 0, 0)
//   NAdam: (mu_(t+1)/(1-P_(t+1)), 1/sqrt(1-b2^t), (1-mu_t)/(1-P_t), 0)
//   RMSprop: (0, 1, 0, 0)
// out receives the four values; returns P_t (NAdam; the input otherwise).
inline double opt_coefficients(int opt, double b1, double b2, long long t, double p_prev, float out[4]) {
  const double td = (double)t;
  const float inv_sqrt_bc2 = (float)(1.0 / std::sqrt(1.0 - std::pow(b2, td)));
  out[2] = out[3] = 0.f;
  if (opt == FPM_OPT_NADAM) {
    const double mt = nadam_mu(b1, td), mn = nadam_mu(b1, td + 1.0);
    const double pt = p_prev * mt, pn = pt * mn;
    out[0] = (float)(mn / (1.0 - pn));
    out[1] = inv_sqrt_bc2;
    out[2] = (float)((1.0 - mt) / (1.0 - pt));
    return pt;
  }
  if (opt == FPM_OPT_RMSPROP) {
    out[0] = 0.f;
    out[1] = 1.f;
    return p_prev;
  }
  out[0] = (float)(1.0 / (1.0 - std::pow(b1, td)));
  out[1] = inv_sqrt_bc2;
  return p_prev;
}

}  // namespace fpmk
