// Nonlocal projector step in mixed precision (Eq. pauli_ks, D |beta><beta|):
// becp = beta^H psi, D-scaling, hpsi += beta (D becp), with FP32 operands and
// FP32 accumulation on the CUDA cores; the FP64 input bands are rounded to FP32
// on the way in and the FP32 result is added to the FP64 output.
#include <algorithm>

#include "common.cuh"
#include "gemm.cuh"

namespace pwh {

__global__ void k_to_f32(const double2* __restrict__ src, int64_t lds, int64_t npw, int nb,
                         float2* __restrict__ dst) {
  int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % npw, b = t / npw;
    double2 z = src[b * lds + i];
    dst[t] = make_float2((float)z.x, (float)z.y);
  }
}

__global__ void k_add_f32(const float2* __restrict__ src, int64_t npw, int nb,
                          double2* __restrict__ dst, int64_t ldd) {
  int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % npw, b = t / npw;
    float2 z = src[t];
    double2 h = dst[b * ldd + i];
    dst[b * ldd + i] = make_double2(h.x + (double)z.x, h.y + (double)z.y);
  }
}

__global__ void k_d_to_f32(const double2* __restrict__ src, int64_t n, float2* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = make_float2((float)src[t].x, (float)src[t].y);
}

void prepare_tc_projectors(System& s) { (void)s; }

void nonlocal_mixed(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
                    cudaStream_t st) {
  if (s.nproj == 0 || nb <= 0) return;
  const int P = s.nproj;
  const int64_t n = s.npw * (int64_t)nb;
  // ws_becp: [psi32 | out32 | becp32 x2 | D32]
  size_t need = (size_t)(2 * n + 2 * (int64_t)P * nb + (s.d_diag ? 0 : (int64_t)P * P)) * sizeof(float2);
  ensure(s.ws_becp, need);
  float2* psi32 = (float2*)s.ws_becp.p;
  float2* out32 = psi32 + n;
  float2* becp = out32 + n;
  float2* becp2 = becp + (size_t)P * nb;
  float2* d32 = becp2 + (size_t)P * nb;
  int g = (int)std::min<int64_t>(152 * 16, (n + 255) / 256);
  k_to_f32<<<g, 256, 0, st>>>(psi, ldp, s.npw, nb, psi32);
  PWH_LAUNCH_CHECK();
  const float2 one = make_float2(1, 0), zero = make_float2(0, 0);
  if (s.d_diag) {
    cgemm<float>(s, true, P, nb, (int)s.npw, one, s.d_beta32, s.npw, psi32, s.npw, zero, becp, P, st,
                 s.d_ddiag);
  } else {
    k_d_to_f32<<<64, 256, 0, st>>>(s.d_dfull, (int64_t)P * P, d32);
    cgemm<float>(s, true, P, nb, (int)s.npw, one, s.d_beta32, s.npw, psi32, s.npw, zero, becp2, P, st);
    cgemm<float>(s, false, P, nb, P, one, d32, P, becp2, P, zero, becp, P, st);
  }
  cgemm<float>(s, false, (int)s.npw, nb, P, one, s.d_beta32, s.npw, becp, P, zero, out32, s.npw, st);
  k_add_f32<<<g, 256, 0, st>>>(out32, s.npw, nb, hpsi, ldh);
  PWH_LAUNCH_CHECK();
}

}  // namespace pwh
