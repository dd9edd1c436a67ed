// Per-problem state of the lockstep IPM (Sec. 5.1 Algorithm run for R problems at once,
// each with its own scalars).  Shared by the lockstep driver (mrhs.cu) and the
// multi-pass partial-DCT operator (large_dct.cu), which reads the stop flags.
#pragma once

#include <stdint.h>

namespace mfipm {

struct Col {
  double tau, cn, mu, sigma, alpha_p, alpha_d, alpha_p1, alpha_d1, mu_t, prev_ap, prev_ad;
  double rel_gap, P_obj, rz0, rz, res2, rho;
  float alpha, beta;
  int stop, active, corr, corr_next, correctors, pcg_iters, ipm_iters, done;
  int64_t nmat;
};

// operator behind the lockstep IPM
enum { OP_SHARED_BF16 = 0, OP_LARGE_DCT = 1 };

// which problems an operator pass works on
enum { GATE_ALL = 0, GATE_ACTIVE = 1, GATE_LIVE = 2 };

}  // namespace mfipm
