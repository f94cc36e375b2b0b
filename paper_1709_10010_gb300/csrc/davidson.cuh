// Block Davidson solver (davidson.cu).
#pragma once
#include "common.cuh"

namespace pwh {
// gamma: real bands at k = 0, psi on the half sphere (gamma_prepare done)
pwh_status davidson_solve(System& s, const pwh_davidson_opts& o, double2* psi, int64_t ldpsi,
                          double* eig, pwh_davidson_stats* stats, bool gamma = false);
}
