// H|psi> = kinetic + local (FFT passes) + nonlocal sum_ij beta_i D_ij <beta_j|psi>
// (Eq. pauli_ks, S = 1), and the public entry points that apply it.
//
// Nonlocal step: becp = beta^H psi (the p_ij of Sec. "New parallelization
// levels"), becp' = D becp, hpsi += beta becp'.  FP64: complex GEMMs on the FP64
// pipe, with a diagonal D folded into the split-K reduction.  Mixed: the BF16
// tensor-core path of gemm_tc.cu.
#include <algorithm>

#include "common.cuh"
#include "gemm.cuh"

namespace pwh {

__global__ void k_permute_in(const double2* __restrict__ src, int64_t lds, int64_t npw, int nb,
                             const int32_t* __restrict__ int_to_pub, double2* __restrict__ dst,
                             int64_t ldd) {
  int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % npw, b = t / npw;
    dst[b * ldd + i] = src[b * lds + int_to_pub[i]];
  }
}

__global__ void k_permute_out(const double2* __restrict__ src, int64_t lds, int64_t npw, int nb,
                              const int32_t* __restrict__ int_to_pub, double2* __restrict__ dst,
                              int64_t ldd) {
  int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % npw, b = t / npw;
    dst[b * ldd + int_to_pub[i]] = src[b * lds + i];
  }
}

static int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(152 * 16, (n + 255) / 256));
}

void permute_public_to_internal(System& s, const double2* src, double2* dst, int nb, int64_t lds) {
  const int64_t n = s.npw * (int64_t)nb;
  k_permute_in<<<grid_for(n), 256, 0, s.stream>>>(src, lds > 0 ? lds : s.npw, s.npw, nb,
                                                  s.d_int_to_pub, dst, s.npw);
  PWH_LAUNCH_CHECK();
}

void nonlocal_fp64(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
                   cudaStream_t st) {
  if (s.nproj == 0 || nb <= 0) return;
  const int P = s.nproj;
  ensure(s.ws_becp, (size_t)2 * P * nb * sizeof(double2));
  double2* becp = (double2*)s.ws_becp.p;
  double2* becp2 = becp + (size_t)P * nb;
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  if (s.d_diag) {
    cgemm<double>(s, true, P, nb, (int)s.npw, one, s.d_beta64, s.npw, psi, ldp, zero, becp, P, st,
                  s.d_ddiag);
  } else {
    cgemm<double>(s, true, P, nb, (int)s.npw, one, s.d_beta64, s.npw, psi, ldp, zero, becp2, P, st);
    cgemm<double>(s, false, P, nb, P, one, s.d_dfull, P, becp2, P, zero, becp, P, st);
  }
  cgemm<double>(s, false, (int)s.npw, nb, P, one, s.d_beta64, s.npw, becp, P, one, hpsi, ldh, st);
}

void ace_apply(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
               int precision);  // exx.cu

void apply_internal(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
                    int precision) {
  if (!s.have_v) throw Error{PWH_ERR_STATE, "pwh_set_potential has not been called"};
  if (nb <= 0) return;
  if (precision == PWH_FP64) {
    local_kinetic<double>(s, nb, psi, ldp, hpsi, ldh, s.stream);
    nonlocal_fp64(s, nb, psi, ldp, hpsi, ldh, s.stream);
    ace_apply(s, nb, psi, ldp, hpsi, ldh, precision);
  } else {
    // the nonlocal term first, into an FP32 buffer that the last FFT pass adds
    float2* vnl = nullptr;
    if (s.nproj > 0) {
      ensure(s.ws_vnl, (size_t)s.npw * nb * sizeof(float2));
      vnl = (float2*)s.ws_vnl.p;
      nonlocal_mixed(s, nb, psi, ldp, vnl, s.npw, s.stream, precision == PWH_MIXED_FAST ? 1 : 3);
    }
    local_kinetic<float>(s, nb, psi, ldp, hpsi, ldh, s.stream, vnl, s.npw);
    ace_apply(s, nb, psi, ldp, hpsi, ldh, precision);
  }
}

}  // namespace pwh

using namespace pwh;

extern "C" {

pwh_status pwh_apply_h_internal(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi,
                                void* hpsi, int64_t ld_hpsi) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CHECK_ARG(nb >= 0, "nb < 0");
    if (nb == 0) return;
    PWH_CHECK_ARG(psi && hpsi, "null band pointer");
    PWH_CHECK_ARG(ld_psi >= s.npw && ld_hpsi >= s.npw, "leading dimension < npw");
    apply_internal(s, nb, (const double2*)psi, ld_psi, (double2*)hpsi, ld_hpsi, s.precision);
  });
}

pwh_status pwh_apply_h(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi, void* hpsi,
                       int64_t ld_hpsi) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CHECK_ARG(nb >= 0, "nb < 0");
    if (nb == 0) return;
    PWH_CHECK_ARG(psi && hpsi, "null band pointer");
    PWH_CHECK_ARG(ld_psi >= s.npw && ld_hpsi >= s.npw, "leading dimension < npw");
    if (!s.have_v) throw Error{PWH_ERR_STATE, "pwh_set_potential has not been called"};
    const size_t n = (size_t)s.npw * nb;
    ensure(s.ws_psi, n * sizeof(double2));
    ensure(s.ws_hpsi, n * sizeof(double2));
    double2* pi = (double2*)s.ws_psi.p;
    double2* hi = (double2*)s.ws_hpsi.p;
    k_permute_in<<<grid_for(n), 256, 0, s.stream>>>((const double2*)psi, ld_psi, s.npw, nb,
                                                    s.d_int_to_pub, pi, s.npw);
    PWH_LAUNCH_CHECK();
    apply_internal(s, nb, pi, s.npw, hi, s.npw, s.precision);
    k_permute_out<<<grid_for(n), 256, 0, s.stream>>>(hi, s.npw, s.npw, nb, s.d_int_to_pub,
                                                     (double2*)hpsi, ld_hpsi);
    PWH_LAUNCH_CHECK();
  });
}

pwh_status pwh_apply_h_host(pwh_system* sys, int32_t nb, const void* psi_host, void* hpsi_host) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CHECK_ARG(nb >= 0, "nb < 0");
    if (nb == 0) return;
    PWH_CHECK_ARG(psi_host && hpsi_host, "null band pointer");
    const size_t n = (size_t)s.npw * nb;
    // ws_host holds the device copies of psi (first half) and hpsi (second half)
    ensure(s.ws_host, 2 * n * sizeof(double2));
    double2* dp = (double2*)s.ws_host.p;
    double2* dh = dp + n;
    PWH_CUDA(cudaMemcpyAsync(dp, psi_host, n * sizeof(double2), cudaMemcpyHostToDevice, s.stream));
    pwh_status st = pwh_apply_h(sys, nb, dp, s.npw, dh, s.npw);
    if (st != PWH_OK) throw Error{st, pwh_last_error()};
    PWH_CUDA(cudaMemcpyAsync(hpsi_host, dh, n * sizeof(double2), cudaMemcpyDeviceToHost, s.stream));
    PWH_CUDA(cudaStreamSynchronize(s.stream));
  });
}

}  // extern "C"
