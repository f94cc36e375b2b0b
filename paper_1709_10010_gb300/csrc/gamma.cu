// Real bands at the Gamma point (k = 0): half-sphere storage and two real bands
// per complex transform (the real-wavefunction trick of the Gamma-only codes
// named in Sec. "Advanced implementation of exact (Fock) exchange" and Sec.
// "Many-body perturbation theory").
//
// A real psi(r) has c(-G) = conj c(G); the half sphere (G = 0 and every G whose
// first nonzero Miller index is positive) carries it.  H is complex-linear, so
// for two real bands psi_1, psi_2 and Psi = psi_1 + i psi_2 on the full sphere,
// H Psi = H psi_1 + i H psi_2; when H maps real functions to real functions
// (real V(r), beta(-G) = conj beta(G), real D) both terms are conjugate
// symmetric and
//     (H psi_1)(G) = (Phi(G) + conj Phi(-G)) / 2,
//     (H psi_2)(G) = (Phi(G) - conj Phi(-G)) / (2i),     Phi = H Psi.
// So nb real bands cost one complex H application of ceil(nb/2) bands: half
// the FFTs, and projector GEMMs of half the width (half the band bytes and
// flops of nb complex bands).  Packing writes Psi in the library's internal
// (stick) order directly, unpacking reads it from there.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "common.cuh"

namespace pwh {

void apply_internal(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
                    int precision);

// Psi_j at the internal positions of G and -G from half-sphere bands 2j, 2j+1
// (band 2j+1 absent for the last pair of an odd nb); c(0) keeps its real part,
// times f0 (sqrt 2 for bands stored with c(0) / sqrt 2, else 1).
__global__ void k_gamma_pack(const double2* __restrict__ psi, int64_t ldp, int64_t nh, int nb,
                             const int32_t* __restrict__ pos, const int32_t* __restrict__ neg,
                             double2* __restrict__ dst, int64_t npw, double f0) {
  const int np = (nb + 1) / 2;
  const int64_t tot = nh * np;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t h = t % nh;
    const int j = (int)(t / nh);
    const double2 a = psi[(size_t)(2 * j) * ldp + h];
    const double2 b = 2 * j + 1 < nb ? psi[(size_t)(2 * j + 1) * ldp + h] : make_double2(0.0, 0.0);
    const int32_t ip = pos[h], in = neg[h];
    double2* d = dst + (size_t)j * npw;
    if (ip == in) {
      d[ip] = make_double2(f0 * a.x, f0 * b.x);
    } else {
      d[ip] = make_double2(a.x - b.y, a.y + b.x);  // a + i b
      d[in] = make_double2(a.x + b.y, b.x - a.y);  // conj(a) + i conj(b)
    }
  }
}

// H psi_{2j}, H psi_{2j+1} on the half sphere from Phi_j = H Psi_j (internal
// order); the G = 0 results times g0 (1 / sqrt 2 for the scaled storage).
__global__ void k_gamma_unpack(const double2* __restrict__ phi, int64_t npw, int64_t nh, int nb,
                               const int32_t* __restrict__ pos, const int32_t* __restrict__ neg,
                               double2* __restrict__ out, int64_t ldo, double g0) {
  const int np = (nb + 1) / 2;
  const int64_t tot = nh * np;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t h = t % nh;
    const int j = (int)(t / nh);
    const double2* f = phi + (size_t)j * npw;
    const int32_t ip = pos[h], in = neg[h];
    const double2 p = f[ip], n = f[in];
    if (ip == in) {
      out[(size_t)(2 * j) * ldo + h] = make_double2(g0 * p.x, 0.0);
      if (2 * j + 1 < nb) out[(size_t)(2 * j + 1) * ldo + h] = make_double2(g0 * p.y, 0.0);
    } else {
      out[(size_t)(2 * j) * ldo + h] = make_double2(0.5 * (p.x + n.x), 0.5 * (p.y - n.y));
      if (2 * j + 1 < nb)
        out[(size_t)(2 * j + 1) * ldo + h] = make_double2(0.5 * (p.y + n.y), -0.5 * (p.x - n.x));
    }
  }
}

// Largest |beta_p(-G) - conj beta_p(G)| and largest |beta_p(G)| over the half
// sphere, as FP32 bit patterns (non-negative floats order like their bits).
__global__ void k_gamma_beta_check(const double2* __restrict__ beta, int64_t npw, int64_t nh,
                                   int nproj, const int32_t* __restrict__ pos,
                                   const int32_t* __restrict__ neg, unsigned* __restrict__ out) {
  float dmax = 0.f, bmax = 0.f;
  const int64_t tot = nh * nproj;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t h = t % nh;
    const int64_t p = t / nh;
    const double2 a = beta[p * npw + pos[h]], b = beta[p * npw + neg[h]];
    dmax = fmaxf(dmax, (float)hypot(b.x - a.x, b.y + a.y));
    bmax = fmaxf(bmax, (float)hypot(a.x, a.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, __float_as_uint(dmax));
    atomicMax(out + 1, __float_as_uint(bmax));
  }
}

// Largest |Im D_ij| and largest |D_ij| of the full D, same encoding.
__global__ void k_gamma_d_check(const double2* __restrict__ D, int64_t n, unsigned* __restrict__ out) {
  float imax = 0.f, dmax = 0.f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    imax = fmaxf(imax, (float)fabs(D[t].y));
    dmax = fmaxf(dmax, (float)hypot(D[t].x, D[t].y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    imax = fmaxf(imax, __shfl_xor_sync(0xffffffffu, imax, o));
    dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out + 2, __float_as_uint(imax));
    atomicMax(out + 3, __float_as_uint(dmax));
  }
}

static int gamma_grid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(152 * 16, (n + 255) / 256));
}

// The half sphere and its internal positions (built on first use).
static void gamma_maps(System& s) {
  if (s.d_gam_pos) return;
  for (int d = 0; d < 3; ++d)
    if (s.kpoint[d] != 0.0) throw Error{PWH_ERR_ARG, "real bands need k = 0"};
  const int64_t npw = s.npw;
  std::vector<int32_t> pub_to_int(npw);
  for (int64_t i = 0; i < npw; ++i) pub_to_int[s.int_to_pub[i]] = (int32_t)i;
  auto key = [](int a, int b, int c) {
    return ((int64_t)(a + 1024) << 22) | ((int64_t)(b + 1024) << 11) | (int64_t)(c + 1024);
  };
  std::unordered_map<int64_t, int32_t> where;
  where.reserve((size_t)npw * 2);
  for (int64_t g = 0; g < npw; ++g)
    where[key(s.miller[3 * g], s.miller[3 * g + 1], s.miller[3 * g + 2])] = (int32_t)g;
  std::vector<int32_t> pub, pos, neg, shell;
  std::vector<double> kin;
  int64_t g0 = -1;
  for (int64_t g = 0; g < npw; ++g) {
    const int m1 = s.miller[3 * g], m2 = s.miller[3 * g + 1], m3 = s.miller[3 * g + 2];
    const bool half = m1 > 0 || (m1 == 0 && (m2 > 0 || (m2 == 0 && m3 >= 0)));
    if (!half) continue;
    auto it = where.find(key(-m1, -m2, -m3));
    if (it == where.end()) throw Error{PWH_ERR_ARG, "the sphere is not symmetric under G -> -G"};
    if (m1 == 0 && m2 == 0 && m3 == 0) g0 = (int64_t)pub.size();
    pub.push_back((int32_t)g);
    pos.push_back(pub_to_int[g]);
    neg.push_back(pub_to_int[it->second]);
    kin.push_back(s.kin_pub[g]);
    shell.push_back(s.shell_pub[g]);
  }
  const size_t nh = pub.size();
  // one allocation: pos, neg, shell (int32), then the kinetic energies (8-byte aligned)
  const size_t ints = (3 * nh + 1) & ~(size_t)1;
  int32_t* d = nullptr;
  PWH_CUDA(cudaMalloc((void**)&d, ints * sizeof(int32_t) + nh * sizeof(double)));
  double* dk = (double*)(d + ints);
  PWH_CUDA(cudaMemcpyAsync(d, pos.data(), nh * sizeof(int32_t), cudaMemcpyHostToDevice, s.stream));
  PWH_CUDA(cudaMemcpyAsync(d + nh, neg.data(), nh * sizeof(int32_t), cudaMemcpyHostToDevice,
                           s.stream));
  PWH_CUDA(cudaMemcpyAsync(d + 2 * nh, shell.data(), nh * sizeof(int32_t), cudaMemcpyHostToDevice,
                           s.stream));
  PWH_CUDA(cudaMemcpyAsync(dk, kin.data(), nh * sizeof(double), cudaMemcpyHostToDevice, s.stream));
  PWH_CUDA(cudaStreamSynchronize(s.stream));
  s.gam_pub = std::move(pub);
  s.d_gam_pos = d;
  s.d_gam_neg = d + nh;
  s.d_gam_shell = d + 2 * nh;
  s.d_gam_kin = dk;
  s.gam_g0 = g0;
}

// Whether the projectors keep real functions real (checked once per set).
static void gamma_check_projectors(System& s) {
  if (s.nproj == 0 || s.gam_proj_ok == 1) return;
  if (s.gam_proj_ok == 0)
    throw Error{PWH_ERR_ARG, "projectors break G -> -G conjugate symmetry or D is not real"};
  const int64_t nh = (int64_t)s.gam_pub.size();
  unsigned* d = nullptr;
  PWH_CUDA(cudaMalloc((void**)&d, 4 * sizeof(unsigned)));
  PWH_CUDA(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), s.stream));
  k_gamma_beta_check<<<gamma_grid(nh * s.nproj), 256, 0, s.stream>>>(
      s.d_beta64, s.npw, nh, s.nproj, s.d_gam_pos, s.d_gam_neg, d);
  cudaError_t e = cudaGetLastError();
  note_launch();
  if (e == cudaSuccess && !s.d_diag) {
    const int64_t n = (int64_t)s.nproj * s.nproj;
    k_gamma_d_check<<<gamma_grid(n), 256, 0, s.stream>>>(s.d_dfull, n, d);
    e = cudaGetLastError();
    note_launch();
  }
  unsigned h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
  cudaFree(d);
  PWH_CUDA(e);
  float v[4];
  for (int i = 0; i < 4; ++i) std::memcpy(&v[i], &h[i], sizeof(float));
  // FP64 projectors of real functions agree to rounding; 1e-10 leaves room
  // for projectors generated through a different formula for -G
  const bool ok = v[0] <= 1e-10f * v[1] && v[2] <= 1e-12f * v[3];
  s.gam_proj_ok = ok ? 1 : 0;
  if (!ok) throw Error{PWH_ERR_ARG, "projectors break G -> -G conjugate symmetry or D is not real"};
}

// Whether the ACE projectors (when set) are real functions, so that the ACE
// term keeps real bands real (checked once per pwh_set_ace).
static void gamma_check_ace(System& s) {
  if (s.ace_n == 0 || s.ace_real == 1) return;
  if (s.ace_real == 0) throw Error{PWH_ERR_ARG, "the ACE projectors are not real functions"};
  const int64_t nh = (int64_t)s.gam_pub.size();
  unsigned* d = nullptr;
  PWH_CUDA(cudaMalloc((void**)&d, 4 * sizeof(unsigned)));
  PWH_CUDA(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), s.stream));
  k_gamma_beta_check<<<gamma_grid(nh * s.ace_n), 256, 0, s.stream>>>(
      s.d_ace, s.npw, nh, s.ace_n, s.d_gam_pos, s.d_gam_neg, d);
  cudaError_t e = cudaGetLastError();
  note_launch();
  unsigned h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
  cudaFree(d);
  PWH_CUDA(e);
  float v[2];
  for (int i = 0; i < 2; ++i) std::memcpy(&v[i], &h[i], sizeof(float));
  s.ace_real = v[0] <= 1e-10f * v[1] ? 1 : 0;
  if (!s.ace_real) throw Error{PWH_ERR_ARG, "the ACE projectors are not real functions"};
}

void gamma_prepare(System& s) {
  gamma_maps(s);
  gamma_check_projectors(s);
  gamma_check_ace(s);
}

void gamma_apply(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
                 int precision, bool scaled0) {
  if (nb <= 0) return;
  const int64_t nh = (int64_t)s.gam_pub.size();
  const int np = (nb + 1) / 2;
  const size_t n = (size_t)s.npw * np;
  ensure(s.ws_psi, n * sizeof(double2));
  ensure(s.ws_hpsi, n * sizeof(double2));
  double2* pi = (double2*)s.ws_psi.p;
  double2* hi = (double2*)s.ws_hpsi.p;
  const double r2 = 1.4142135623730951;  // sqrt 2
  k_gamma_pack<<<gamma_grid(nh * np), 256, 0, s.stream>>>(psi, ldp, nh, nb, s.d_gam_pos, s.d_gam_neg,
                                                         pi, s.npw, scaled0 ? r2 : 1.0);
  PWH_LAUNCH_CHECK();
  apply_internal(s, np, pi, s.npw, hi, s.npw, precision);
  k_gamma_unpack<<<gamma_grid(nh * np), 256, 0, s.stream>>>(hi, s.npw, nh, nb, s.d_gam_pos,
                                                           s.d_gam_neg, hpsi, ldh,
                                                           scaled0 ? 1.0 / r2 : 1.0);
  PWH_LAUNCH_CHECK();
}

}  // namespace pwh

using namespace pwh;

extern "C" {

pwh_status pwh_get_gamma_half(pwh_system* sys, int64_t* npw_half, int32_t* pub_index) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    gamma_maps(s);
    if (npw_half) *npw_half = (int64_t)s.gam_pub.size();
    if (pub_index) std::memcpy(pub_index, s.gam_pub.data(), s.gam_pub.size() * sizeof(int32_t));
  });
}

pwh_status pwh_apply_h_gamma(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi,
                             void* hpsi, int64_t ld_hpsi) {
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CHECK_ARG(nb >= 0, "nb < 0");
    gamma_maps(s);
    const int64_t nh = (int64_t)s.gam_pub.size();
    if (nb == 0) return;
    PWH_CHECK_ARG(psi && hpsi, "null band pointer");
    PWH_CHECK_ARG(ld_psi >= nh && ld_hpsi >= nh, "leading dimension < npw_half");
    if (!s.have_v) throw Error{PWH_ERR_STATE, "pwh_set_potential has not been called"};
    gamma_check_projectors(s);
    gamma_check_ace(s);
    gamma_apply(s, nb, (const double2*)psi, ld_psi, (double2*)hpsi, ld_hpsi, s.precision, false);
  });
}

}  // extern "C"
