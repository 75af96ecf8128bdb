// Outcome codes of the device-resident CG loop and their mapping to the C ABI's
// hqmc_status (plain C++: the host-only status test compiles this header alone).
#pragma once

#include "hqmc.h"

#if defined(__CUDACC__)
#define HQMC_HOST_DEVICE __host__ __device__
#else
#define HQMC_HOST_DEVICE
#endif

namespace hqmc {

// CG_REC_CONVERGED: the recursive residual met tol; the true residual still has
// to be checked.  CG_CONVERGED: the true FP64 residual met tol.
// CG_STAGNATED (mixed solver): eight reliable updates cut the true residual by
// less than 2x, i.e. FP32 rounding stalls the recurrence on this field.  (Plain
// CG on these ill-conditioned fields may gain less than 10x in 200 iterations,
// so a tighter test would abandon FP32 on healthy solves.)
enum { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXIT = 2, CG_BREAKDOWN = 3, CG_NONFINITE = 4, CG_REC_CONVERGED = 5,
       CG_STAGNATED = 6 };

// Status of a solve that left the loop in state `done`.  `timed_out`: a bounded
// device-side wait gave up during the solve (the kernel that waited poisons its
// outputs with NaN, so the loop itself ends as CG_NONFINITE or worse); that
// cause is reported in preference to the symptom.
HQMC_HOST_DEVICE inline int solve_status(int done, bool timed_out) {
  if (timed_out) return HQMC_ETIMEOUT;
  switch (done) {
    case CG_CONVERGED: return HQMC_OK;
    case CG_MAXIT: return HQMC_ENOTCONV;
    case CG_BREAKDOWN: return HQMC_EBREAKDOWN;
    case CG_STAGNATED: return HQMC_ENOTCONV;
    default: return HQMC_ENONFINITE;  // CG_NONFINITE, or a loop that ended in no final state
  }
}

}  // namespace hqmc
