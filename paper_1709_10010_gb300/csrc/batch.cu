// Batched eigensolves of many independent systems (cells x k-points), the
// single-GPU counterpart of the paper's pool (k-point) and image levels of
// parallelism (Sec. "New parallelization levels"): a pool of host threads
// drives one block Davidson per system, each system on its own CUDA stream,
// so that the small kernels of many systems run concurrently on the GPU.
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace pwh;

extern "C" pwh_status pwh_batch_davidson_solve(int32_t n, pwh_system* const* systems,
                                               const pwh_davidson_opts* opts, void* const* psi_io,
                                               const int64_t* ld_psi, double* const* eig,
                                               pwh_davidson_stats* stats, pwh_status* status_out,
                                               int32_t nthreads) {
  std::vector<std::string> msgs;
  pwh_status first = PWH_OK;
  pwh_status g = guarded([&] {
    PWH_CHECK_ARG(n >= 0, "n < 0");
    if (n == 0) return;
    PWH_CHECK_ARG(systems && opts && psi_io && ld_psi && eig && status_out, "null argument");
    PWH_CHECK_ARG(nthreads >= 1 && nthreads <= 256, "nthreads out of range [1, 256]");
    for (int i = 0; i < n; ++i) {
      PWH_CHECK_ARG(systems[i] && psi_io[i] && eig[i], "null system, band block or eig");
      for (int j = 0; j < i; ++j)
        PWH_CHECK_ARG(systems[j] != systems[i], "a system appears twice in the batch");
    }
    int dev = 0;
    PWH_CUDA(cudaGetDevice(&dev));
    msgs.assign(n, std::string());
    std::atomic<int> next{0};
    auto worker = [&] {
      cudaSetDevice(dev);
      for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
        status_out[i] = pwh_davidson_solve(systems[i], &opts[i], psi_io[i], ld_psi[i], eig[i],
                                           stats ? &stats[i] : nullptr);
        if (status_out[i] != PWH_OK) msgs[i] = pwh_last_error();
      }
    };
    const int nt = std::min<int>(nthreads, n);
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    for (int i = 0; i < n; ++i)
      if (status_out[i] != PWH_OK && first == PWH_OK) {
        first = status_out[i];
        set_error("system " + std::to_string(i) + ": " + msgs[i]);
      }
  });
  return g != PWH_OK ? g : first;
}
