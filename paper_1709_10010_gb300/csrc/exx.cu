// Exact (Fock) exchange and the adaptively compressed exchange operator (Sec.
// "Advanced implementation of exact (Fock) exchange and hybrid functionals":
// Eq. Vx, the pair-density potentials of Eq. Poisson solved in reciprocal
// space, and ACE, Eq. Vxace).  Hartree atomic units, FP64.
//
//   (V_x phi)(r) = - sum_j f_j psi_j(r) v_j(r),
//   v_j(G) = 4 pi rho_j(G) / |G|^2 (G != 0; the G = 0 term left out),
//   rho_j(r) = conj(psi_j(r)) phi(r).
//
// Every band is put on the full FFT box once (scatter, inverse 3D FFT); for
// each target band the pair densities of a batch of occupied bands are formed,
// transformed, scaled by the Coulomb factor, transformed back and reduced
// into the target's exchange potential times its band, which is transformed
// and gathered on the sphere at the end.  On the alias-free box
// (N_d >= 4 mmax_d + 1) this equals the reciprocal-space sum exactly.  The
// batch is sized to keep its pair boxes within L2.
//
// ACE: xi_i = V_x psi_i, M = psi^H xi; -M = L L^H; zeta = xi L^-H, so that
// sum_jm xi_j (M^-1)_jm <xi_m| = -zeta zeta^H; H then carries -zeta zeta^H psi
// (two GEMMs on the tensor-core paths of the system's precision).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "dense.cuh"
#include "gemm.cuh"

namespace pwh {

static int exx_grid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(152 * 16, (n + 255) / 256));
}

// box[b][idx[g]] = c[b * ld + g] for nb bands (boxes zeroed before)
__global__ void k_exx_scatter(const double2* __restrict__ c, int64_t ld, int64_t npw, int nb,
                              const int32_t* __restrict__ idx, double2* __restrict__ box,
                              int64_t nbox) {
  const int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = t % npw, b = t / npw;
    box[b * nbox + idx[g]] = c[b * ld + g];
  }
}

// pair[j][r] = conj(U[j][r]) P[r] for J boxes of nbox points
__global__ void k_exx_pair(const double2* __restrict__ U, const double2* __restrict__ P,
                           double2* __restrict__ pair, int64_t nbox, int J) {
  const int64_t tot = nbox * J;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t % nbox;
    const double2 u = U[t], p = P[r];
    pair[t] = make_double2(u.x * p.x + u.y * p.y, u.x * p.y - u.y * p.x);
  }
}

// pair[j][G] *= kern[G] (the Coulomb factor with the transform normalisation)
__global__ void k_exx_coulomb(double2* __restrict__ pair, const double* __restrict__ kern,
                              int64_t nbox, int J) {
  const int64_t tot = nbox * J;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double k = kern[t % nbox];
    pair[t] = make_double2(k * pair[t].x, k * pair[t].y);
  }
}

// W[r] -= sum_j f_j U[j][r] v[j][r] (one writer per point, fixed order over j)
__global__ void k_exx_acc(const double2* __restrict__ U, const double2* __restrict__ v,
                          const double* __restrict__ f, double2* __restrict__ W, int64_t nbox,
                          int J) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nbox;
       r += (int64_t)gridDim.x * blockDim.x) {
    double2 w = W[r];
    for (int j = 0; j < J; ++j) {
      const double2 u = U[(size_t)j * nbox + r], a = v[(size_t)j * nbox + r];
      w.x -= f[j] * (u.x * a.x - u.y * a.y);
      w.y -= f[j] * (u.x * a.y + u.y * a.x);
    }
    W[r] = w;
  }
}

// W[j][r] -= f_i U_i[r] conj(v[j][r]) for the J boxes of a batch, skipping
// box jskip: the term of source i in the exchange of band j, from the pair
// potential of (i, j) (v_ji = conj(v_ij), the Coulomb kernel being real)
__global__ void k_exx_acc_t(const double2* __restrict__ Ui, const double2* __restrict__ v,
                            double fi, double2* __restrict__ W, int64_t nbox, int J, int jskip) {
  const int64_t tot = nbox * J;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / nbox);
    if (j == jskip) continue;
    const int64_t r = t - (int64_t)j * nbox;
    const double2 u = Ui[r], a = v[t];
    // u conj(a)
    W[t].x -= fi * (u.x * a.x + u.y * a.y);
    W[t].y -= fi * (u.y * a.x - u.x * a.y);
  }
}

// out[g] = scale * box[idx[g]]
__global__ void k_exx_gather(const double2* __restrict__ box, const int32_t* __restrict__ idx,
                             int64_t npw, double scale, double2* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < npw;
       g += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = box[idx[g]];
    out[g] = make_double2(scale * v.x, scale * v.y);
  }
}

// dst[:, j] = src[int_to_pub[i], j] (public -> internal order), k columns
__global__ void k_exx_perm_in(const double2* __restrict__ src, int64_t lds, int64_t npw, int k,
                              const int32_t* __restrict__ i2p, double2* __restrict__ dst) {
  const int64_t tot = npw * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % npw, j = t / npw;
    dst[j * npw + i] = src[j * lds + i2p[i]];
  }
}

// S = -(M + M^H) / 2 (k x k): the Gram matrix whose Cholesky factor gives ACE
__global__ void k_exx_neg_herm(const double2* __restrict__ M, int k, double2* __restrict__ S) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += gridDim.x * blockDim.x) {
    const int i = t % k, j = t / k;
    const double2 a = M[(size_t)j * k + i], b = M[(size_t)i * k + j];
    S[t] = make_double2(-0.5 * (a.x + b.x), -0.5 * (a.y - b.y));
  }
}

// ------------------------------------------------------------------ host ----
// Full-box index of each public plane wave (C order, i3 fastest) and the
// Coulomb factor on the box (built on first use, uploaded once).
static void exx_tables(System& s) {
  if (s.d_boxidx) return;
  const int64_t npw = s.npw, nbox = (int64_t)s.n1 * s.n2 * s.n3;
  std::vector<int32_t> idx(npw);
  for (int64_t g = 0; g < npw; ++g) {
    const int i1 = ((s.miller[3 * g] % s.n1) + s.n1) % s.n1;
    const int i2 = ((s.miller[3 * g + 1] % s.n2) + s.n2) % s.n2;
    const int i3 = ((s.miller[3 * g + 2] % s.n3) + s.n3) % s.n3;
    idx[g] = (int32_t)(((int64_t)i1 * s.n2 + i2) * s.n3 + i3);
  }
  // reciprocal vectors b_j (rows) with a_i . b_j = 2 pi delta_ij: 2 pi (A^-1)^T
  const double* a = s.lattice;
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  const double c = 2.0 * M_PI / det;
  const double b[9] = {c * (a[4] * a[8] - a[5] * a[7]), c * (a[5] * a[6] - a[3] * a[8]),
                       c * (a[3] * a[7] - a[4] * a[6]), c * (a[2] * a[7] - a[1] * a[8]),
                       c * (a[0] * a[8] - a[2] * a[6]), c * (a[1] * a[6] - a[0] * a[7]),
                       c * (a[1] * a[5] - a[2] * a[4]), c * (a[2] * a[3] - a[0] * a[5]),
                       c * (a[0] * a[4] - a[1] * a[3])};
  const double scale = 4.0 * M_PI / (std::fabs(det) * (double)nbox);
  std::vector<double> kern(nbox);
  const int n[3] = {s.n1, s.n2, s.n3};
  for (int i1 = 0; i1 < s.n1; ++i1)
    for (int i2 = 0; i2 < s.n2; ++i2)
      for (int i3 = 0; i3 < s.n3; ++i3) {
        const int m[3] = {i1 > n[0] / 2 ? i1 - n[0] : i1, i2 > n[1] / 2 ? i2 - n[1] : i2,
                          i3 > n[2] / 2 ? i3 - n[2] : i3};
        double g2 = 0.0;
        for (int x = 0; x < 3; ++x) {
          const double gx = m[0] * b[0 + x] + m[1] * b[3 + x] + m[2] * b[6 + x];
          g2 += gx * gx;
        }
        kern[((int64_t)i1 * s.n2 + i2) * s.n3 + i3] = g2 > 0.0 ? scale / g2 : 0.0;
      }
  PWH_CUDA(cudaMalloc((void**)&s.d_boxidx, npw * sizeof(int32_t)));
  PWH_CUDA(cudaMalloc((void**)&s.d_kern, nbox * sizeof(double)));
  PWH_CUDA(cudaMemcpyAsync(s.d_boxidx, idx.data(), npw * sizeof(int32_t), cudaMemcpyHostToDevice,
                           s.stream));
  PWH_CUDA(cudaMemcpyAsync(s.d_kern, kern.data(), nbox * sizeof(double), cudaMemcpyHostToDevice,
                           s.stream));
  PWH_CUDA(cudaStreamSynchronize(s.stream));
}

// Device scratch freed at scope exit (after the stream has drained).
struct ExxScratch {
  cudaStream_t st;
  std::vector<void*> p;
  void* get(size_t bytes) {
    void* q = nullptr;
    PWH_CUDA(cudaMalloc(&q, std::max<size_t>(bytes, 256)));
    p.push_back(q);
    return q;
  }
  ~ExxScratch() {
    cudaStreamSynchronize(st);
    for (void* q : p) cudaFree(q);
  }
};

// out[:, i] = V_x phi_i for nb bands (public order, device), occupied bands
// psi_occ (public order, device) with host weights occ.
static void exx_apply(System& s, int nocc, const double2* psi_occ, int64_t ld_occ,
                      const double* occ, int nb, const double2* phi, int64_t ld_phi, double2* out,
                      int64_t ld_out) {
  exx_tables(s);
  cudaStream_t st = s.stream;
  const int64_t npw = s.npw, nbox = (int64_t)s.n1 * s.n2 * s.n3;
  const size_t bb = (size_t)nbox * sizeof(double2);
  // occupied bands per batch: their pair boxes within about 64 MB
  const int J = (int)std::max<int64_t>(1, std::min<int64_t>(nocc, ((int64_t)64 << 20) / (int64_t)bb));
  ExxScratch sc{st, {}};
  double2* U = (double2*)sc.get(bb * nocc);
  double2* pair = (double2*)sc.get(bb * J);
  double2* P = (double2*)sc.get(bb);
  double2* W = (double2*)sc.get(bb);
  double* f = (double*)sc.get(nocc * sizeof(double));
  PWH_CUDA(cudaMemcpyAsync(f, occ, nocc * sizeof(double), cudaMemcpyHostToDevice, st));
  // the occupied bands on the box
  PWH_CUDA(cudaMemsetAsync(U, 0, bb * nocc, st));
  k_exx_scatter<<<exx_grid(npw * nocc), 256, 0, st>>>(psi_occ, ld_occ, npw, nocc, s.d_boxidx, U,
                                                     nbox);
  PWH_LAUNCH_CHECK();
  box_fft(s, U, true, nocc, nbox);
  for (int i = 0; i < nb; ++i) {
    PWH_CUDA(cudaMemsetAsync(P, 0, bb, st));
    PWH_CUDA(cudaMemsetAsync(W, 0, bb, st));
    k_exx_scatter<<<exx_grid(npw), 256, 0, st>>>(phi + (size_t)i * ld_phi, ld_phi, npw, 1,
                                                s.d_boxidx, P, nbox);
    PWH_LAUNCH_CHECK();
    box_fft(s, P, true);
    for (int j0 = 0; j0 < nocc; j0 += J) {
      const int jb = std::min(J, nocc - j0);
      const double2* Uj = U + (size_t)j0 * nbox;
      k_exx_pair<<<exx_grid(nbox * jb), 256, 0, st>>>(Uj, P, pair, nbox, jb);
      PWH_LAUNCH_CHECK();
      box_fft(s, pair, false, jb, nbox);
      k_exx_coulomb<<<exx_grid(nbox * jb), 256, 0, st>>>(pair, s.d_kern, nbox, jb);
      PWH_LAUNCH_CHECK();
      box_fft(s, pair, true, jb, nbox);
      k_exx_acc<<<exx_grid(nbox), 256, 0, st>>>(Uj, pair, f + j0, W, nbox, jb);
      PWH_LAUNCH_CHECK();
    }
    box_fft(s, W, false);
    k_exx_gather<<<exx_grid(npw), 256, 0, st>>>(W, s.d_boxidx, npw, 1.0 / (double)nbox,
                                               out + (size_t)i * ld_out);
    PWH_LAUNCH_CHECK();
  }
}

// out[:, i] = V_x psi_i for the occupied bands themselves: each unordered pair
// (i, j) is transformed once and feeds both bands' exchange, so about half the
// pair densities of exx_apply with the same bands as targets.
static void exx_apply_self(System& s, int nocc, const double2* psi, int64_t ld, const double* occ,
                           double2* out, int64_t ld_out) {
  exx_tables(s);
  cudaStream_t st = s.stream;
  const int64_t npw = s.npw, nbox = (int64_t)s.n1 * s.n2 * s.n3;
  const size_t bb = (size_t)nbox * sizeof(double2);
  const int J = (int)std::max<int64_t>(1, std::min<int64_t>(nocc, ((int64_t)64 << 20) / (int64_t)bb));
  ExxScratch sc{st, {}};
  double2* U = (double2*)sc.get(bb * nocc);
  double2* W = (double2*)sc.get(bb * nocc);
  double2* pair = (double2*)sc.get(bb * J);
  double* f = (double*)sc.get(nocc * sizeof(double));
  PWH_CUDA(cudaMemcpyAsync(f, occ, nocc * sizeof(double), cudaMemcpyHostToDevice, st));
  PWH_CUDA(cudaMemsetAsync(U, 0, bb * nocc, st));
  PWH_CUDA(cudaMemsetAsync(W, 0, bb * nocc, st));
  k_exx_scatter<<<exx_grid(npw * nocc), 256, 0, st>>>(psi, ld, npw, nocc, s.d_boxidx, U, nbox);
  PWH_LAUNCH_CHECK();
  box_fft(s, U, true, nocc, nbox);
  for (int i = 0; i < nocc; ++i) {
    const double2* Ui = U + (size_t)i * nbox;
    double2* Wi = W + (size_t)i * nbox;
    for (int j0 = 0; j0 <= i; j0 += J) {
      const int jb = std::min(J, i + 1 - j0);
      const double2* Uj = U + (size_t)j0 * nbox;
      k_exx_pair<<<exx_grid(nbox * jb), 256, 0, st>>>(Uj, Ui, pair, nbox, jb);
      PWH_LAUNCH_CHECK();
      box_fft(s, pair, false, jb, nbox);
      k_exx_coulomb<<<exx_grid(nbox * jb), 256, 0, st>>>(pair, s.d_kern, nbox, jb);
      PWH_LAUNCH_CHECK();
      box_fft(s, pair, true, jb, nbox);
      // band i: sources j0.. (v_ij); bands j0.. (j < i): source i (conj v_ij)
      k_exx_acc<<<exx_grid(nbox), 256, 0, st>>>(Uj, pair, f + j0, Wi, nbox, jb);
      PWH_LAUNCH_CHECK();
      k_exx_acc_t<<<exx_grid(nbox * jb), 256, 0, st>>>(Ui, pair, occ[i], W + (size_t)j0 * nbox,
                                                      nbox, jb, i - j0 < jb ? i - j0 : -1);
      PWH_LAUNCH_CHECK();
    }
  }
  box_fft(s, W, false, nocc, nbox);
  for (int i = 0; i < nocc; ++i) {
    k_exx_gather<<<exx_grid(npw), 256, 0, st>>>(W + (size_t)i * nbox, s.d_boxidx, npw,
                                               1.0 / (double)nbox, out + (size_t)i * ld_out);
    PWH_LAUNCH_CHECK();
  }
}

void ace_apply(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
               int precision) {
  if (s.ace_n == 0 || nb <= 0) return;
  ensure(s.ws_ace, (size_t)s.ace_n * nb * sizeof(double2));
  double2* T = (double2*)s.ws_ace.p;
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0), mone = make_double2(-1, 0);
  const int npw = (int)s.npw, k = s.ace_n;
  if (precision == PWH_FP64) {
    cgemm<double>(s, true, k, nb, npw, one, s.d_ace, npw, psi, ldp, zero, T, k, s.stream);
    cgemm<double>(s, false, npw, nb, k, mone, s.d_ace, npw, T, k, one, hpsi, ldh, s.stream);
  } else {
    cgemm_f32(s, true, k, nb, npw, one, s.d_ace, npw, psi, ldp, zero, T, k, s.stream);
    cgemm_f32(s, false, npw, nb, k, mone, s.d_ace, npw, T, k, one, hpsi, ldh, s.stream);
  }
}

}  // namespace pwh

using namespace pwh;

extern "C" {

pwh_status pwh_exx_apply(pwh_system* sys, int32_t nocc, const void* psi_occ, int64_t ld_occ,
                         const double* occ, int32_t nb, const void* phi, int64_t ld_phi, void* out,
                         int64_t ld_out) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CHECK_ARG(nocc >= 1 && nb >= 0, "nocc < 1 or nb < 0");
    if (nb == 0) return;
    PWH_CHECK_ARG(psi_occ && occ && phi && out, "null argument");
    PWH_CHECK_ARG(ld_occ >= s.npw && ld_phi >= s.npw && ld_out >= s.npw,
                  "leading dimension < npw");
    for (int j = 0; j < nocc; ++j) PWH_CHECK_ARG(std::isfinite(occ[j]), "non-finite weight");
    exx_apply(s, nocc, (const double2*)psi_occ, ld_occ, occ, nb, (const double2*)phi, ld_phi,
              (double2*)out, ld_out);
    PWH_CUDA(cudaStreamSynchronize(s.stream));
  });
}

pwh_status pwh_set_ace(pwh_system* sys, int32_t nocc, const void* psi_occ, int64_t ld_occ,
                       const double* occ, double alpha, int32_t* rank) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CHECK_ARG(nocc >= 0 && nocc <= 1024 && nocc <= s.npw, "nocc out of range [0, min(1024, npw)]");
    PWH_CUDA(cudaStreamSynchronize(s.stream));
    if (s.d_ace) cudaFree(s.d_ace);
    s.d_ace = nullptr;
    s.ace_n = 0;
    s.ace_real = -1;
    if (rank) *rank = 0;
    if (nocc == 0) return;
    PWH_CHECK_ARG(psi_occ && occ, "null argument");
    PWH_CHECK_ARG(ld_occ >= s.npw, "ld_occ < npw");
    PWH_CHECK_ARG(std::isfinite(alpha) && alpha > 0.0, "alpha must be > 0");
    for (int j = 0; j < nocc; ++j)
      PWH_CHECK_ARG(std::isfinite(occ[j]) && occ[j] > 0.0, "occupations must be > 0");
    cudaStream_t st = s.stream;
    const int64_t npw = s.npw;
    ExxScratch sc{st, {}};
    double2* xi = (double2*)sc.get((size_t)npw * nocc * sizeof(double2));
    double2* M = (double2*)sc.get((size_t)nocc * nocc * sizeof(double2));
    double2* S = (double2*)sc.get((size_t)nocc * nocc * sizeof(double2));
    double2* Tr = (double2*)sc.get((size_t)nocc * nocc * sizeof(double2));
    double2* zeta = (double2*)sc.get((size_t)npw * nocc * sizeof(double2));
    int* kk = (int*)sc.get(sizeof(int));
    const double2* psi = (const double2*)psi_occ;
    // xi = V_x psi, M = psi^H xi, -M = L L^H with Tr = L^-H (Tr^H (-M) Tr = I)
    exx_apply_self(s, nocc, psi, ld_occ, occ, xi, npw);
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    cgemm<double>(s, true, nocc, nocc, (int)npw, one, psi, ld_occ, xi, npw, zero, M, nocc, st);
    k_exx_neg_herm<<<exx_grid((int64_t)nocc * nocc), 256, 0, st>>>(M, nocc, S);
    PWH_LAUNCH_CHECK();
    DenseWs dw;
    cholqr_factor(s, dw, S, nocc, nullptr, 0.0, Tr, kk, st, false);
    int h_kk = 0;
    PWH_CUDA(cudaMemcpyAsync(&h_kk, kk, sizeof(int), cudaMemcpyDeviceToHost, st));
    PWH_CUDA(cudaStreamSynchronize(st));
    if (h_kk == 0) throw Error{PWH_ERR_ARG, "the exchange matrix of the occupied bands is singular"};
    // zeta = sqrt(alpha) xi Tr (kept columns), then the internal plane-wave order
    cgemm<double>(s, false, (int)npw, h_kk, nocc, make_double2(std::sqrt(alpha), 0.0), xi, npw, Tr,
                  nocc, zero, zeta, npw, st);
    PWH_CUDA(cudaMalloc((void**)&s.d_ace, (size_t)npw * h_kk * sizeof(double2)));
    k_exx_perm_in<<<exx_grid(npw * h_kk), 256, 0, st>>>(zeta, npw, npw, h_kk, s.d_int_to_pub,
                                                       s.d_ace);
    PWH_LAUNCH_CHECK();
    PWH_CUDA(cudaStreamSynchronize(st));
    s.ace_n = h_kk;
    if (rank) *rank = h_kk;
  });
}

}  // extern "C"
