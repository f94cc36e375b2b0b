// Block Davidson solver (davidson.cu).
#pragma once
#include "common.cuh"

namespace pwh {
pwh_status davidson_solve(System& s, const pwh_davidson_opts& o, double2* psi, int64_t ldpsi,
                          double* eig, pwh_davidson_stats* stats);
}
