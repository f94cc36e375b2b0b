// The overlap operator of ultrasoft / PAW projectors and the generalised
// eigenproblem H x = e S x (the S of Eq. pauli_ks, Sec. "Fully relativistic
// projector augmented-wave method"), in the separable form over the
// projectors of the nonlocal term:
//
//   S = 1 + sum_ij |beta_i> q_ij <beta_j|       (q Hermitian, S > 0).
//
// S psi = psi + beta (q (beta^H psi)) reuses the projector products of the
// nonlocal term.  The eigensolvers solve the generalised problem through the
// Loewdin form H' = S^-1/2 H S^-1/2 (same spectrum, eigenvectors
// x = S^-1/2 phi, S-orthonormal), with S^-1/2 separable as well:
// S^-1/2 = 1 + beta K beta^H.  K is built once per pwh_set_overlap from
// G = beta^H beta = W diag(g) W^H (directions with g <= 1e-12 max g carry no
// projector and are left out), M = g^1/2 W^H q W g^1/2 = U diag(mu) U^H and
// K = W g^-1/2 U diag((1 + mu)^-1/2 - 1) U^H g^-1/2 W^H: on the span of the
// projectors, in the orthonormal basis beta W g^-1/2, S is 1 + M; on the
// complement S is the identity.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "gemm.cuh"

namespace pwh {

static int ov_grid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(152 * 16, (n + 255) / 256));
}

// full P x P q from P real diagonal values
__global__ void k_ov_diag_full(const double* __restrict__ d, int P, double2* __restrict__ q) {
  const int64_t tot = (int64_t)P * P;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % P), j = (int)(t / P);
    q[t] = make_double2(i == j ? d[i] : 0.0, 0.0);
  }
}

// Winv[:, c] = W[:, c] g_c^-1/2 and Wsq[:, c] = W[:, c] g_c^1/2 for g_c above
// thr, zero columns otherwise (those directions carry no projector)
__global__ void k_ov_scale_w(const double2* __restrict__ W, const double* __restrict__ g, int P,
                             double thr, double2* __restrict__ Winv, double2* __restrict__ Wsq) {
  const int64_t tot = (int64_t)P * P;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / P);
    const double gc = g[c];
    const bool keep = gc > thr;
    const double a = keep ? 1.0 / sqrt(gc) : 0.0, b = keep ? sqrt(gc) : 0.0;
    Winv[t] = make_double2(a * W[t].x, a * W[t].y);
    Wsq[t] = make_double2(b * W[t].x, b * W[t].y);
  }
}

// Y = diag(f) X^H with f_k = (1 + mu_k)^-1/2 - 1 (P x P); bad[0] = 1 when some
// 1 + mu_k <= 0 (S not positive definite)
__global__ void k_ov_fxh(const double2* __restrict__ X, const double* __restrict__ mu, int P,
                         double2* __restrict__ Y, int* __restrict__ bad) {
  const int64_t tot = (int64_t)P * P;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % P), j = (int)(t / P);
    const double m = mu[i];
    if (!(1.0 + m > 0.0)) {
      if (j == 0) *bad = 1;
      Y[t] = make_double2(0.0, 0.0);
      continue;
    }
    const double f = 1.0 / sqrt(1.0 + m) - 1.0;
    const double2 x = X[(size_t)i * P + j];  // (X^H)_ij = conj(X_ji)
    Y[t] = make_double2(f * x.x, -f * x.y);
  }
}

// Y = X^H (P x P)
__global__ void k_ov_adjoint(const double2* __restrict__ X, int P, double2* __restrict__ Y) {
  const int64_t tot = (int64_t)P * P;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % P), j = (int)(t / P);
    const double2 x = X[(size_t)i * P + j];
    Y[t] = make_double2(x.x, -x.y);
  }
}

// M <- (M + M^H) / 2 (P x P)
__global__ void k_ov_hermitize(double2* __restrict__ M, int P) {
  const int64_t tot = (int64_t)P * P;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % P), j = (int)(t / P);
    if (i > j) continue;
    const double2 a = M[(size_t)j * P + i], b = M[(size_t)i * P + j];
    const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    M[(size_t)j * P + i] = h;
    M[(size_t)i * P + j] = make_double2(h.x, -h.y);
  }
}

__global__ void k_ov_copy(const double2* __restrict__ src, int64_t lds, double2* __restrict__ dst,
                          int64_t ldd, int64_t npw, int k) {
  const int64_t tot = npw * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % npw, j = t / npw;
    dst[j * ldd + i] = src[j * lds + i];
  }
}

// out = in + beta (C (beta^H in)) for nb bands in the internal order (in and
// out may be the same array); C: P x P.  FP64 products (the FP64-equivalent
// tensor-core path above its size threshold) or, for a reduced precision,
// FP32-equivalent ones.
static void sep_apply(System& s, const double2* C, int nb, const double2* in, int64_t ldi,
                      double2* out, int64_t ldo, int prec) {
  if (nb <= 0) return;
  const int P = s.nproj, npw = (int)s.npw;
  cudaStream_t st = s.stream;
  ensure(s.ws_ov, (size_t)2 * P * nb * sizeof(double2));
  double2* b1 = (double2*)s.ws_ov.p;
  double2* b2 = b1 + (size_t)P * nb;
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  if (out != in) {
    k_ov_copy<<<ov_grid((int64_t)npw * nb), 256, 0, st>>>(in, ldi, out, ldo, npw, nb);
    PWH_LAUNCH_CHECK();
  }
  if (prec == PWH_FP64) {
    cgemm<double>(s, true, P, nb, npw, one, s.d_beta64, npw, in, ldi, zero, b1, P, st);
    cgemm<double>(s, false, P, nb, P, one, C, P, b1, P, zero, b2, P, st);
    cgemm<double>(s, false, npw, nb, P, one, s.d_beta64, npw, b2, P, one, out, ldo, st);
  } else {
    cgemm_f32(s, true, P, nb, npw, one, s.d_beta64, npw, in, ldi, zero, b1, P, st);
    cgemm_f32(s, false, P, nb, P, one, C, P, b1, P, zero, b2, P, st);
    cgemm_f32(s, false, npw, nb, P, one, s.d_beta64, npw, b2, P, one, out, ldo, st);
  }
}

void overlap_apply_s(System& s, int nb, const double2* in, int64_t ldi, double2* out, int64_t ldo,
                     int prec) {
  sep_apply(s, s.d_q, nb, in, ldi, out, ldo, prec);
}

void overlap_inv_sqrt(System& s, int nb, const double2* in, int64_t ldi, double2* out,
                      int64_t ldo, int prec) {
  sep_apply(s, s.d_ksq, nb, in, ldi, out, ldo, prec);
}

__global__ void k_ov_perm(const double2* __restrict__ src, int64_t lds, int64_t npw, int nb,
                          const int32_t* __restrict__ i2p, double2* __restrict__ dst, int64_t ldd,
                          int to_public) {
  const int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % npw, b = t / npw;
    if (to_public)
      dst[b * ldd + i2p[i]] = src[b * lds + i];
    else
      dst[b * ldd + i] = src[b * lds + i2p[i]];
  }
}

// K of S^-1/2 = 1 + beta K beta^H from q and the projectors (see the top of
// this file).  Returns false when S is not positive definite.
static bool build_inv_sqrt(System& s) {
  const int P = s.nproj;
  const int64_t npw = s.npw;
  cudaStream_t st = s.stream;
  const size_t mat = (size_t)P * P * sizeof(double2);
  std::vector<void*> bufs;
  auto get = [&](size_t bytes) {
    void* p = nullptr;
    PWH_CUDA(cudaMalloc(&p, std::max<size_t>(bytes, 256)));
    bufs.push_back(p);
    return p;
  };
  struct Free {
    std::vector<void*>& b;
    cudaStream_t st;
    ~Free() {
      cudaStreamSynchronize(st);
      for (void* p : b) cudaFree(p);
    }
  } fr{bufs, st};
  double2* G = (double2*)get(mat);
  double2* W = (double2*)get(mat);
  double2* Winv = (double2*)get(mat);
  double2* Wsq = (double2*)get(mat);
  double2* T = (double2*)get(mat);
  double2* M = (double2*)get(mat);
  double2* U = (double2*)get(mat);
  double* g = (double*)get(P * sizeof(double));
  double* mu = (double*)get(P * sizeof(double));
  int* bad = (int*)get(sizeof(int));
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  const int gr = ov_grid((int64_t)P * P);
  DenseWs dw;
  // G = beta^H beta = W diag(g) W^H
  cgemm<double>(s, true, P, P, (int)npw, one, s.d_beta64, npw, s.d_beta64, npw, zero, G, P, st);
  k_ov_hermitize<<<gr, 256, 0, st>>>(G, P);
  PWH_LAUNCH_CHECK();
  jacobi_eigh(s, dw, G, P, P, P, g, W, st);
  std::vector<double> hg(P);
  PWH_CUDA(cudaMemcpyAsync(hg.data(), g, P * sizeof(double), cudaMemcpyDeviceToHost, st));
  PWH_CUDA(cudaStreamSynchronize(st));
  const double gmax = *std::max_element(hg.begin(), hg.end());
  k_ov_scale_w<<<gr, 256, 0, st>>>(W, g, P, 1e-12 * gmax, Winv, Wsq);
  PWH_LAUNCH_CHECK();
  // M = g^1/2 W^H q W g^1/2 = U diag(mu) U^H
  cgemm<double>(s, false, P, P, P, one, s.d_q, P, Wsq, P, zero, T, P, st);
  cgemm<double>(s, true, P, P, P, one, Wsq, P, T, P, zero, M, P, st);
  k_ov_hermitize<<<gr, 256, 0, st>>>(M, P);
  PWH_LAUNCH_CHECK();
  jacobi_eigh(s, dw, M, P, P, P, mu, U, st);
  // F = U diag((1 + mu)^-1/2 - 1) U^H (into G), K = (W g^-1/2) F (W g^-1/2)^H
  PWH_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_ov_fxh<<<gr, 256, 0, st>>>(U, mu, P, T, bad);
  PWH_LAUNCH_CHECK();
  cgemm<double>(s, false, P, P, P, one, U, P, T, P, zero, G, P, st);
  cgemm<double>(s, false, P, P, P, one, Winv, P, G, P, zero, T, P, st);
  k_ov_adjoint<<<gr, 256, 0, st>>>(Winv, P, M);
  PWH_LAUNCH_CHECK();
  cgemm<double>(s, false, P, P, P, one, T, P, M, P, zero, s.d_ksq, P, st);
  k_ov_hermitize<<<gr, 256, 0, st>>>(s.d_ksq, P);
  PWH_LAUNCH_CHECK();
  int h_bad = 0;
  PWH_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PWH_CUDA(cudaStreamSynchronize(st));
  return h_bad == 0;
}

}  // namespace pwh

using namespace pwh;

extern "C" {

pwh_status pwh_set_overlap(pwh_system* sys, const void* q, int32_t q_is_diag, int32_t on_device) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CUDA(cudaStreamSynchronize(s.stream));
    for (double2** p : {&s.d_q, &s.d_ksq}) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
    s.have_overlap = false;
    if (!q) return;
    if (s.nproj == 0) throw Error{PWH_ERR_STATE, "the overlap needs projectors (pwh_set_projectors)"};
    const int P = s.nproj;
    const size_t mat = (size_t)P * P * sizeof(double2);
    PWH_CUDA(cudaMalloc((void**)&s.d_q, mat));
    PWH_CUDA(cudaMalloc((void**)&s.d_ksq, mat));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (q_is_diag) {
      double* d = nullptr;
      PWH_CUDA(cudaMalloc((void**)&d, P * sizeof(double)));
      cudaError_t e = cudaMemcpyAsync(d, q, P * sizeof(double), kind, s.stream);
      if (e == cudaSuccess) {
        k_ov_diag_full<<<ov_grid((int64_t)P * P), 256, 0, s.stream>>>(d, P, s.d_q);
        e = cudaGetLastError();
        note_launch();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
      cudaFree(d);
      PWH_CUDA(e);
    } else {
      PWH_CUDA(cudaMemcpyAsync(s.d_q, q, mat, kind, s.stream));
      k_ov_hermitize<<<ov_grid((int64_t)P * P), 256, 0, s.stream>>>(s.d_q, P);
      PWH_LAUNCH_CHECK();
    }
    if (!build_inv_sqrt(s)) {
      for (double2** p : {&s.d_q, &s.d_ksq}) {
        cudaFree(*p);
        *p = nullptr;
      }
      throw Error{PWH_ERR_ARG, "S = 1 + beta q beta^H is not positive definite"};
    }
    s.have_overlap = true;
  });
}

pwh_status pwh_apply_s(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi, void* spsi,
                       int64_t ld_spsi) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CHECK_ARG(nb >= 0, "nb < 0");
    if (nb == 0) return;
    PWH_CHECK_ARG(psi && spsi, "null band pointer");
    PWH_CHECK_ARG(ld_psi >= s.npw && ld_spsi >= s.npw, "leading dimension < npw");
    const size_t n = (size_t)s.npw * nb;
    ensure(s.ws_psi, n * sizeof(double2));
    ensure(s.ws_hpsi, n * sizeof(double2));
    double2* pi = (double2*)s.ws_psi.p;
    double2* so = (double2*)s.ws_hpsi.p;
    k_ov_perm<<<ov_grid((int64_t)n), 256, 0, s.stream>>>((const double2*)psi, ld_psi, s.npw, nb,
                                                        s.d_int_to_pub, pi, s.npw, 0);
    PWH_LAUNCH_CHECK();
    if (s.have_overlap) {
      overlap_apply_s(s, nb, pi, s.npw, so, s.npw, PWH_FP64);
    } else {
      k_ov_copy<<<ov_grid((int64_t)n), 256, 0, s.stream>>>(pi, s.npw, so, s.npw, s.npw, nb);
      PWH_LAUNCH_CHECK();
    }
    k_ov_perm<<<ov_grid((int64_t)n), 256, 0, s.stream>>>(so, s.npw, s.npw, nb, s.d_int_to_pub,
                                                        (double2*)spsi, ld_spsi, 1);
    PWH_LAUNCH_CHECK();
  });
}

}  // extern "C"
