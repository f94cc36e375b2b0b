// The self-consistent-field steps either side of H|psi>: the electron density
// of a set of bands, and the new local potential V_LOC = v_ion + V_H + v_xc
// (the Kohn-Sham equations solved to self-consistency, Sec. "Introduction";
// the Hartree potential by the Fourier-space Poisson solution on the FFT box,
// as for the pair densities of exact exchange, Sec. "Advanced implementation
// of exact (Fock) exchange").  Hartree atomic units, FP64 throughout.
//
//   rho(r) = sum_n f_n |psi_n(r)|^2,  psi_n(r) = Omega^{-1/2} sum_G c_n(G) e^{i(k+G).r}
//   V_H(G) = 4 pi rho(G) / |G|^2 (G != 0; G = 0 and Nyquist planes dropped)
//   LDA: Slater exchange and the Perdew-Zunger (Phys. Rev. B 23, 5048, 1981)
//        parametrisation of the Ceperley-Alder correlation energy
#include <cmath>

#include "common.cuh"

namespace pwh {

// Perdew-Zunger constants (unpolarised gas, Hartree units)
constexpr double kPzG = -0.1423, kPzB1 = 1.0529, kPzB2 = 0.3334;
constexpr double kPzA = 0.0311, kPzB = -0.048, kPzC = 0.0020, kPzD = -0.0116;
constexpr double kRhoMin = 1e-20;

__device__ __forceinline__ void lda_point(double rho, double& exc, double& vxc) {
  if (!(rho > kRhoMin)) {
    exc = 0.0;
    vxc = 0.0;
    return;
  }
  const double pi = 3.14159265358979323846;
  const double rs = cbrt(3.0 / (4.0 * pi * rho));
  const double ex = -0.75 * cbrt(3.0 * rho / pi);
  const double vx = 4.0 / 3.0 * ex;
  double ec, vc;
  if (rs >= 1.0) {
    const double sq = sqrt(rs);
    const double den = 1.0 + kPzB1 * sq + kPzB2 * rs;
    ec = kPzG / den;
    vc = ec * (1.0 + 7.0 / 6.0 * kPzB1 * sq + 4.0 / 3.0 * kPzB2 * rs) / den;
  } else {
    const double lr = log(rs);
    ec = kPzA * lr + kPzB + kPzC * rs * lr + kPzD * rs;
    vc = kPzA * lr + (kPzB - kPzA / 3.0) + 2.0 / 3.0 * kPzC * rs * lr + (2.0 * kPzD - kPzC) / 3.0 * rs;
  }
  exc = ex + ec;
  vxc = vx + vc;
}

// rho (C order) -> complex box
__global__ void k_real_to_box(const double* __restrict__ rho, int64_t n, double2* __restrict__ box) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    box[t] = make_double2(rho[t], 0.0);
}

// box = N^3 rho(G) in -> V_H(G) = 4 pi rho(G) / |G|^2 (m_d read as m_d - N_d
// above N_d / 2; G = 0 and Nyquist planes zeroed)
__global__ void k_poisson(double2* __restrict__ box, int n1, int n2, int n3, const double* __restrict__ b9) {
  const int64_t tot = (int64_t)n1 * n2 * n3;
  const double inv_n = 1.0 / (double)tot, fourpi = 4.0 * 3.14159265358979323846;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(t % n3), i2 = (int)((t / n3) % n2), i1 = (int)(t / ((int64_t)n2 * n3));
    const bool nyq = ((n1 % 2 == 0) && i1 == n1 / 2) || ((n2 % 2 == 0) && i2 == n2 / 2) ||
                     ((n3 % 2 == 0) && i3 == n3 / 2);
    const double m1 = i1 > n1 / 2 ? i1 - n1 : i1, m2 = i2 > n2 / 2 ? i2 - n2 : i2,
                 m3 = i3 > n3 / 2 ? i3 - n3 : i3;
    const double gx = m1 * b9[0] + m2 * b9[3] + m3 * b9[6];
    const double gy = m1 * b9[1] + m2 * b9[4] + m3 * b9[7];
    const double gz = m1 * b9[2] + m2 * b9[5] + m3 * b9[8];
    const double g2 = gx * gx + gy * gy + gz * gz;
    const double f = (nyq || !(g2 > 0.0)) ? 0.0 : fourpi * inv_n / g2;
    const double2 v = box[t];
    box[t] = make_double2(v.x * f, v.y * f);
  }
}

// v_out = v_ion + V_H + v_xc; en[0] += sum V_H rho, en[1] += sum rho eps_xc,
// en[2] += sum rho v_xc (fixed-order block partials, one atomic a block)
__global__ void k_xc_combine(const double* __restrict__ rho, const double2* __restrict__ vh,
                             const double* __restrict__ v_ion, int64_t n, double* __restrict__ v_out,
                             double* __restrict__ en) {
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double r = rho[t];
    double exc, vxc;
    lda_point(r, exc, vxc);
    const double h = vh[t].x;
    v_out[t] = (v_ion ? v_ion[t] : 0.0) + h + vxc;
    a0 += h * r;
    a1 += r * exc;
    a2 += r * vxc;
  }
  __shared__ double red[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a0;
    red[1][threadIdx.x >> 5] = a1;
    red[2][threadIdx.x >> 5] = a2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
      s2 += red[2][w];
    }
    atomicAdd(en, s0);
    atomicAdd(en + 1, s1);
    atomicAdd(en + 2, s2);
  }
}

// internal layout [i3][i2][i1] -> C order [i1][i2][i3], times scale
__global__ void k_grid_to_c(const double* __restrict__ in, int n1, int n2, int n3, double scale,
                            double* __restrict__ out) {
  const int64_t tot = (int64_t)n1 * n2 * n3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(t % n3), i2 = (int)((t / n3) % n2), i1 = (int)(t / ((int64_t)n2 * n3));
    out[t] = scale * in[((size_t)i3 * n2 + i2) * n1 + i1];
  }
}

static int grid1(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(152 * 8, (n + 255) / 256)); }

static double cell_volume(const System& s) {
  const double* a = s.lattice;
  return std::fabs(a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                   a[2] * (a[3] * a[7] - a[4] * a[6]));
}

}  // namespace pwh

using namespace pwh;

extern "C" pwh_status pwh_density(pwh_system* sys, int32_t nb, const void* psi, int64_t ld_psi,
                                  const double* occ, double* rho) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && rho, "null argument");
    System& s = sys->s;
    PWH_CHECK_ARG(nb >= 0, "nb < 0");
    PWH_CHECK_ARG(nb == 0 || (psi && occ), "null band block or occupations");
    PWH_CHECK_ARG(nb == 0 || ld_psi >= s.npw, "ld_psi < npw");
    const int64_t ng = (int64_t)s.n1 * s.n2 * s.n3;
    const size_t need = (size_t)ng * sizeof(double) + (size_t)nb * sizeof(double) + 256;
    ensure(s.ws_grid, need);
    double* acc = (double*)s.ws_grid.p;
    double* occ_dev = acc + ng;
    cudaStream_t st = s.stream;
    PWH_CUDA(cudaMemsetAsync(acc, 0, ng * sizeof(double), st));
    if (nb > 0) {
      PWH_CUDA(cudaMemcpyAsync(occ_dev, occ, nb * sizeof(double), cudaMemcpyHostToDevice, st));
      ensure(s.ws_psi, (size_t)s.npw * nb * sizeof(double2));
      double2* pi = (double2*)s.ws_psi.p;
      permute_public_to_internal(s, (const double2*)psi, pi, nb, ld_psi);
      density_accumulate(s, nb, pi, occ_dev, acc);
    }
    k_grid_to_c<<<grid1(ng), 256, 0, st>>>(acc, s.n1, s.n2, s.n3, 1.0 / cell_volume(s), rho);
    PWH_LAUNCH_CHECK();
    // the host occupations must outlive the copy
    PWH_CUDA(cudaStreamSynchronize(st));
  });
}

extern "C" pwh_status pwh_hartree_xc(pwh_system* sys, const double* rho, const double* v_ion,
                                     double* v_out, double* energies) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && rho && v_out, "null argument");
    System& s = sys->s;
    const int64_t ng = (int64_t)s.n1 * s.n2 * s.n3;
    ensure(s.ws_grid, (size_t)ng * sizeof(double2) + 16 * sizeof(double) + 256);
    double2* box = (double2*)s.ws_grid.p;
    double* en = (double*)(box + ng);
    double* b9 = en + 4;
    cudaStream_t st = s.stream;
    // reciprocal vectors b_i (rows), a_i . b_j = 2 pi delta_ij
    const double* a = s.lattice;
    const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                       a[2] * (a[3] * a[7] - a[4] * a[6]);
    const double tp = 2.0 * 3.14159265358979323846 / det;
    double bh[9] = {tp * (a[4] * a[8] - a[5] * a[7]), tp * (a[5] * a[6] - a[3] * a[8]), tp * (a[3] * a[7] - a[4] * a[6]),
                    tp * (a[2] * a[7] - a[1] * a[8]), tp * (a[0] * a[8] - a[2] * a[6]), tp * (a[1] * a[6] - a[0] * a[7]),
                    tp * (a[1] * a[5] - a[2] * a[4]), tp * (a[2] * a[3] - a[0] * a[5]), tp * (a[0] * a[4] - a[1] * a[3])};
    PWH_CUDA(cudaMemcpyAsync(b9, bh, sizeof(bh), cudaMemcpyHostToDevice, st));
    PWH_CUDA(cudaMemsetAsync(en, 0, 3 * sizeof(double), st));
    k_real_to_box<<<grid1(ng), 256, 0, st>>>(rho, ng, box);
    PWH_LAUNCH_CHECK();
    box_fft(s, box, false);                      // N^3 rho(G)
    k_poisson<<<grid1(ng), 256, 0, st>>>(box, s.n1, s.n2, s.n3, b9);
    PWH_LAUNCH_CHECK();
    box_fft(s, box, true);                       // V_H(r)
    k_xc_combine<<<grid1(ng), 256, 0, st>>>(rho, box, v_ion, ng, v_out, en);
    PWH_LAUNCH_CHECK();
    double eh[3];
    PWH_CUDA(cudaMemcpyAsync(eh, en, sizeof(eh), cudaMemcpyDeviceToHost, st));
    PWH_CUDA(cudaStreamSynchronize(st));
    const double dv = cell_volume(s) / (double)ng;
    if (energies) {
      energies[0] = 0.5 * eh[0] * dv;
      energies[1] = eh[1] * dv;
      energies[2] = eh[2] * dv;
    }
  });
}
