// Learned preconditioner (not in the paper; the learned part of this library):
// a 4 -> 64 -> 64 -> 1 SiLU network s = MLP(f) corrects the Teter-Payne-Allan
// diagonal per (shell of equal |k+G|, band):  K = K_TPA(x) * exp(clip(s, -3, 3)).
//
//  * features/targets of (shell, band) rows from Ritz vectors X, their H X,
//    Ritz values and the converged bands X* (training data harvested from the
//    solver's own trajectories);
//  * forward, loss + backward (block-level weight-gradient reduction), Adam;
//  * the per-iteration factors used by the eigensolver's preconditioner.
//
// Parameter vector (FP32): W1 (64x4 row-major), b1, W2 (64x64), b2, W3 (64), b3,
// then 8 floats of feature ranges (min f1..f4, max f1..f4) outside which the
// preconditioner falls back to plain TPA (s = 0).
#include <algorithm>
#include <mutex>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"

namespace pwh {

constexpr int MH = 64, MIN = 4;
constexpr int kMlpParams = MH * MIN + MH + MH * MH + MH + MH + 1;  // 4545
constexpr int kMlpBlob = kMlpParams + 8;

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_g(float z) {
  const float sg = 1.f / (1.f + __expf(-z));
  return sg * (1.f + z * (1.f - sg));
}

// Load the parameters into shared memory (all threads).
__device__ void mlp_load(const float* __restrict__ p, float* sp) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sp[i] = p[i];
  __syncthreads();
}

// Forward pass of one row; optional caches of pre-activations.
__device__ float mlp_row(const float* sp, const float f[4], float* z1c, float* z2c) {
  const float* W1 = sp;
  const float* b1 = W1 + MH * MIN;
  const float* W2 = b1 + MH;
  const float* b2 = W2 + MH * MH;
  const float* W3 = b2 + MH;
  const float b3 = W3[MH];
  float h1[MH];
#pragma unroll 8
  for (int i = 0; i < MH; ++i) {
    float z = b1[i] + W1[i * 4] * f[0] + W1[i * 4 + 1] * f[1] + W1[i * 4 + 2] * f[2] +
              W1[i * 4 + 3] * f[3];
    if (z1c) z1c[i] = z;
    h1[i] = silu_f(z);
  }
  float s = b3;
  for (int i = 0; i < MH; ++i) {
    float z = b2[i];
#pragma unroll 16
    for (int j = 0; j < MH; ++j) z += W2[i * MH + j] * h1[j];
    if (z2c) z2c[i] = z;
    s += W3[i] * silu_f(z);
  }
  return s;
}

__global__ void k_mlp_forward(const float* __restrict__ p, const float* __restrict__ F, int64_t rows,
                              float* __restrict__ s) {
  extern __shared__ float sp[];
  mlp_load(p, sp);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    float f[4] = {F[4 * r], F[4 * r + 1], F[4 * r + 2], F[4 * r + 3]};
    s[r] = mlp_row(sp, f, nullptr, nullptr);
  }
}

// Loss sum w (s - y)^2 / wsum and its gradient, accumulated (atomically) into
// g (kMlpParams) and loss[0].  128 rows per block; the block reduces the
// weight gradients of its rows in shared memory before one atomic per weight.
constexpr int GR = 128;
__global__ void __launch_bounds__(GR) k_mlp_grad(const float* __restrict__ p,
                                                 const float* __restrict__ F,
                                                 const float* __restrict__ y,
                                                 const float* __restrict__ w, int64_t rows,
                                                 float inv_wsum, float* __restrict__ g,
                                                 float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* sp = sm;                      // parameters
  float* sh1 = sp + kMlpParams + 3;    // GR x MH: h1
  float* sd2 = sh1 + GR * MH;          // GR x MH: dz2
  float* sd1 = sd2 + GR * MH;          // GR x MH: dz1
  float* sf = sd1 + GR * MH;           // GR x 4: features
  float* sds = sf + GR * 4;            // GR: ds
  float* sh2 = sds + GR;               // GR x MH: h2 (for gW3)
  mlp_load(p, sp);
  const float* W1 = sp;
  const float* W2 = W1 + MH * MIN + MH;
  const float* W3 = W2 + MH * MH + MH;
  const int64_t r = blockIdx.x * (int64_t)GR + threadIdx.x;
  const int t = threadIdx.x;
  float z1[MH], z2[MH];
  float ds = 0.f;
  float f[4] = {0, 0, 0, 0};
  if (r < rows) {
    f[0] = F[4 * r]; f[1] = F[4 * r + 1]; f[2] = F[4 * r + 2]; f[3] = F[4 * r + 3];
    const float s = mlp_row(sp, f, z1, z2);
    const float e = s - y[r];
    ds = 2.f * w[r] * e * inv_wsum;
    atomicAdd(loss, w[r] * e * e * inv_wsum);
  } else {
    for (int i = 0; i < MH; ++i) z1[i] = z2[i] = 0.f;
  }
  // backward of one row
  for (int i = 0; i < MH; ++i) {
    sh1[t * MH + i] = (r < rows) ? silu_f(z1[i]) : 0.f;
    sh2[t * MH + i] = (r < rows) ? silu_f(z2[i]) : 0.f;
    sd2[t * MH + i] = ds * W3[i] * silu_g(z2[i]);
  }
  for (int j = 0; j < MH; ++j) {
    float acc = 0.f;
    for (int i = 0; i < MH; ++i) acc += sd2[t * MH + i] * W2[i * MH + j];
    sd1[t * MH + j] = acc * silu_g(z1[j]);
  }
  for (int k = 0; k < 4; ++k) sf[t * 4 + k] = f[k];
  sds[t] = ds;
  __syncthreads();
  // block reduction of the weight gradients
  float* gW1 = g;
  float* gb1 = gW1 + MH * MIN;
  float* gW2 = gb1 + MH;
  float* gb2 = gW2 + MH * MH;
  float* gW3 = gb2 + MH;
  float* gb3 = gW3 + MH;
  for (int e = t; e < MH * MH; e += GR) {
    const int i = e / MH, j = e % MH;
    float acc = 0.f;
    for (int q = 0; q < GR; ++q) acc += sd2[q * MH + i] * sh1[q * MH + j];
    atomicAdd(&gW2[e], acc);
  }
  for (int e = t; e < MH * MIN; e += GR) {
    const int i = e / MIN, k = e % MIN;
    float acc = 0.f;
    for (int q = 0; q < GR; ++q) acc += sd1[q * MH + i] * sf[q * 4 + k];
    atomicAdd(&gW1[e], acc);
  }
  for (int i = t; i < MH; i += GR) {
    float a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int q = 0; q < GR; ++q) {
      a1 += sd1[q * MH + i];
      a2 += sd2[q * MH + i];
      a3 += sds[q] * sh2[q * MH + i];
    }
    atomicAdd(&gb1[i], a1);
    atomicAdd(&gb2[i], a2);
    atomicAdd(&gW3[i], a3);
  }
  if (t == 0) {
    float a = 0.f;
    for (int q = 0; q < GR; ++q) a += sds[q];
    atomicAdd(gb3, a);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---------------------------------------------------------- features / data --
__device__ __forceinline__ double tpa_k(double x) {
  const double q = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
  return q / (q + 16.0 * x * x * x * x);
}

__device__ __forceinline__ void make_features(double Tg, double th, double rn, double E, double vbar,
                                              float f[4]) {
  const double x = Tg / E;
  f[0] = (float)log(x + 0.05);
  f[1] = (float)((th - vbar) / E);
  f[2] = (float)fmin(2.0, fmax(-12.0, log10(fmax(rn, 1e-300))));
  f[3] = (float)((Tg + vbar - th) / (Tg + E));
}

// per band: R = HX - X theta (internal order scratch), rn, eref = <x|T|x>/<x|x>;
// per (band, shell): num += Re conj(r) e, den += |r|^2 with e = corrections E.
__global__ void k_shell_stats(const double2* __restrict__ X, const double2* __restrict__ HX,
                              const double2* __restrict__ E, int64_t npw,
                              const double* __restrict__ theta, const int32_t* __restrict__ shell,
                              int nshell, double* __restrict__ num, double* __restrict__ den) {
  const int b = blockIdx.y;
  const double th = theta[b];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npw;
       i += (int64_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * npw + i;
    const double2 x = X[o], hx = HX[o], e = E[o];
    const double rx = hx.x - th * x.x, ry = hx.y - th * x.y;
    const int g = shell[i];
    atomicAdd(&num[(size_t)b * nshell + g], rx * e.x + ry * e.y);
    atomicAdd(&den[(size_t)b * nshell + g], rx * rx + ry * ry);
  }
}

__global__ void k_band_stats(const double2* __restrict__ X, const double2* __restrict__ HX,
                             int64_t npw, const double* __restrict__ theta,
                             const double* __restrict__ kin, double* __restrict__ rn,
                             double* __restrict__ eref) {
  const int b = blockIdx.x;
  const double th = theta[b];
  double s2 = 0, xt = 0, x2 = 0;
  for (int64_t i = threadIdx.x; i < npw; i += blockDim.x) {
    const size_t o = (size_t)b * npw + i;
    const double2 x = X[o], hx = HX[o];
    const double rx = hx.x - th * x.x, ry = hx.y - th * x.y;
    s2 += rx * rx + ry * ry;
    const double a = x.x * x.x + x.y * x.y;
    x2 += a;
    xt += kin[i] * a;
  }
  __shared__ double red[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    xt += __shfl_xor_sync(0xffffffffu, xt, o);
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s2;
    red[1][threadIdx.x >> 5] = xt;
    red[2][threadIdx.x >> 5] = x2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, c = 0, d = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      c += red[1][w];
      d += red[2][w];
    }
    rn[b] = sqrt(a);
    eref[b] = (d > 0 && c > 0) ? c / d : 1.0;
  }
}

// One block per band: features of every shell, target y and weight w.
__global__ void k_make_rows(const double* __restrict__ num, const double* __restrict__ den, int nshell,
                            const double* __restrict__ Tshell, const double* __restrict__ theta,
                            const double* __restrict__ rn, const double* __restrict__ eref,
                            double vbar, float* __restrict__ F, float* __restrict__ y,
                            float* __restrict__ w) {
  const int b = blockIdx.x;
  const double E = eref[b];
  __shared__ double red[2][32];
  double dsum = 0;
  for (int g = threadIdx.x; g < nshell; g += blockDim.x) dsum += den[(size_t)b * nshell + g];
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = dsum;
  __syncthreads();
  double tot = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += red[0][q];
  __syncthreads();
  // raw targets and weights, then the weighted mean
  double wy = 0, ws = 0;
  for (int g = threadIdx.x; g < nshell; g += blockDim.x) {
    const size_t o = (size_t)b * nshell + g;
    const double dn = den[o];
    const double d = dn > 0 ? -num[o] / dn : 0.0;
    const bool ok = d > 0 && dn > 0;
    const double yy = ok ? log(d) - log(tpa_k(Tshell[g] / E)) : 0.0;
    const double ww = ok ? dn / tot : 0.0;
    y[o] = (float)yy;
    w[o] = (float)ww;
    wy += ww * yy;
    ws += ww;
    float f[4];
    make_features(Tshell[g], theta[b], rn[b], E, vbar, f);
    for (int k = 0; k < 4; ++k) F[4 * o + k] = f[k];
  }
  for (int o = 16; o > 0; o >>= 1) {
    wy += __shfl_xor_sync(0xffffffffu, wy, o);
    ws += __shfl_xor_sync(0xffffffffu, ws, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = wy;
    red[1][threadIdx.x >> 5] = ws;
  }
  __syncthreads();
  double mwy = 0, mws = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
    mwy += red[0][q];
    mws += red[1][q];
  }
  const double mean = mws > 0 ? mwy / mws : 0.0;
  for (int g = threadIdx.x; g < nshell; g += blockDim.x) {
    const size_t o = (size_t)b * nshell + g;
    if (w[o] > 0) y[o] = (float)((double)y[o] - mean);
  }
}

// Preconditioner factors for the eigensolver: s[j * nshell + g] for the bands
// idx[j], clipped to [-3, 3], 0 (plain TPA) when a feature leaves the range
// the network was trained on.
__global__ void k_mlp_factors(const float* __restrict__ blob, const int* __restrict__ idx, int k,
                              const double* __restrict__ theta, const double* __restrict__ rn,
                              const double* __restrict__ eref, const double* __restrict__ Tshell,
                              int nshell, double vbar, float* __restrict__ s) {
  extern __shared__ float sp[];
  mlp_load(blob, sp);
  const float* lo = blob + kMlpParams;
  const float* hi = lo + 4;
  const int64_t rows = (int64_t)k * nshell;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(r / nshell), g = (int)(r % nshell);
    const int b = idx[j];
    float f[4];
    make_features(Tshell[g], theta[b], rn[b], eref[b], vbar, f);
    bool inside = true;
    for (int q = 0; q < 4; ++q) inside = inside && f[q] >= lo[q] && f[q] <= hi[q];
    float v = inside ? mlp_row(sp, f, nullptr, nullptr) : 0.f;
    s[r] = fminf(3.f, fmaxf(-3.f, v));
  }
}

static size_t grad_smem() {
  return (size_t)(kMlpParams + 3 + 4 * GR * MH + GR * 4 + GR) * sizeof(float);
}

void mlp_factors(System& s, const int* idx, int k, const double* theta, const double* rn,
                 const double* eref, float* out, cudaStream_t st) {
  const int64_t rows = (int64_t)k * s.nshell;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (rows + 255) / 256));
  k_mlp_factors<<<blocks, 256, kMlpParams * sizeof(float), st>>>(s.d_mlp, idx, k, theta, rn, eref,
                                                                 s.d_Tshell, s.nshell, s.vbar, out);
  PWH_LAUNCH_CHECK();
}

}  // namespace pwh

using namespace pwh;

extern "C" {

pwh_status pwh_mlp_num_params(int32_t* n) {
  return guarded([&] {
    PWH_CHECK_ARG(n, "null argument");
    *n = kMlpBlob;
  });
}

pwh_status pwh_mlp_forward(pwh_system* sys, const float* params, const float* feats, int64_t rows,
                           float* s_out) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && params && feats && s_out, "null argument");
    PWH_CHECK_ARG(rows >= 0, "rows < 0");
    if (rows == 0) return;
    const int blocks = (int)std::min<int64_t>(4096, (rows + 255) / 256);
    k_mlp_forward<<<blocks, 256, kMlpParams * sizeof(float), sys->s.stream>>>(params, feats, rows,
                                                                             s_out);
    PWH_LAUNCH_CHECK();
  });
}

pwh_status pwh_mlp_loss_grad(pwh_system* sys, const float* params, const float* feats,
                             const float* y, const float* w, int64_t rows, double wsum,
                             float* grad_out, float* loss_out) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && params && feats && y && w && grad_out && loss_out, "null argument");
    PWH_CHECK_ARG(rows >= 1 && wsum > 0, "rows >= 1 and wsum > 0 required");
    System& s = sys->s;
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
      cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)grad_smem());
    });
    PWH_CUDA(cudaMemsetAsync(grad_out, 0, kMlpParams * sizeof(float), s.stream));
    PWH_CUDA(cudaMemsetAsync(loss_out, 0, sizeof(float), s.stream));
    const int blocks = (int)((rows + GR - 1) / GR);
    k_mlp_grad<<<blocks, GR, grad_smem(), s.stream>>>(params, feats, y, w, rows, (float)(1.0 / wsum),
                                                      grad_out, loss_out);
    PWH_LAUNCH_CHECK();
  });
}

pwh_status pwh_mlp_adam(pwh_system* sys, float* params, const float* grad, float* m, float* v,
                        int32_t step, float lr) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && params && grad && m && v, "null argument");
    PWH_CHECK_ARG(step >= 1, "step counts from 1");
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
    k_adam<<<32, 256, 0, sys->s.stream>>>(params, grad, m, v, kMlpParams, lr, b1, b2, 1e-8f, c1, c2);
    PWH_LAUNCH_CHECK();
  });
}

pwh_status pwh_mlp_training_rows(pwh_system* sys, int32_t nb, const void* X, const void* HX,
                                 const double* theta, const void* Xstar, float* feats, float* y,
                                 float* w) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && X && HX && theta && Xstar && feats && y && w, "null argument");
    System& s = sys->s;
    PWH_CHECK_ARG(nb >= 1, "nb < 1");
    if (!s.have_v) throw Error{PWH_ERR_STATE, "pwh_set_potential has not been called"};
    const int64_t npw = s.npw;
    cudaStream_t st = s.stream;
    // scratch: internal-order copies of X, HX, X*, corrections E, W (nb x nb), stats
    const size_t nv = (size_t)npw * nb;
    double2* buf = nullptr;
    PWH_CUDA(cudaMalloc((void**)&buf, (4 * nv + (size_t)nb * nb) * sizeof(double2) +
                                          (2 * (size_t)nb * s.nshell + 3 * (size_t)nb) * sizeof(double)));
    double2 *Xi = buf, *HXi = Xi + nv, *Si = HXi + nv, *Ei = Si + nv, *Wm = Ei + nv;
    double* num = (double*)(Wm + (size_t)nb * nb);
    double* den = num + (size_t)nb * s.nshell;
    double* th = den + (size_t)nb * s.nshell;
    double* rn = th + nb;
    double* eref = rn + nb;
    try {
      permute_public_to_internal(s, (const double2*)X, Xi, nb);
      permute_public_to_internal(s, (const double2*)HX, HXi, nb);
      permute_public_to_internal(s, (const double2*)Xstar, Si, nb);
      PWH_CUDA(cudaMemcpyAsync(th, theta, nb * sizeof(double), cudaMemcpyHostToDevice, st));
      // E = X* (X*^H X) - X
      const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
      cgemm<double>(s, true, nb, nb, (int)npw, one, Si, npw, Xi, npw, zero, Wm, nb, st);
      PWH_CUDA(cudaMemcpyAsync(Ei, Xi, nv * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      cgemm<double>(s, false, (int)npw, nb, nb, one, Si, npw, Wm, nb, make_double2(-1, 0), Ei, npw, st);
      PWH_CUDA(cudaMemsetAsync(num, 0, 2 * (size_t)nb * s.nshell * sizeof(double), st));
      dim3 g((unsigned)std::min<int64_t>(64, (npw + 255) / 256), nb);
      k_shell_stats<<<g, 256, 0, st>>>(Xi, HXi, Ei, npw, th, s.d_shell, s.nshell, num, den);
      PWH_LAUNCH_CHECK();
      k_band_stats<<<nb, 256, 0, st>>>(Xi, HXi, npw, th, s.d_kin, rn, eref);
      PWH_LAUNCH_CHECK();
      k_make_rows<<<nb, 256, 0, st>>>(num, den, s.nshell, s.d_Tshell, th, rn, eref, s.vbar, feats, y, w);
      PWH_LAUNCH_CHECK();
      PWH_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      cudaFree(buf);
      throw;
    }
    cudaFree(buf);
  });
}

pwh_status pwh_set_mlp(pwh_system* sys, const float* blob, int32_t n) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && blob, "null argument");
    PWH_CHECK_ARG(n == kMlpBlob, "parameter blob has the wrong length");
    System& s = sys->s;
    if (!s.d_mlp) PWH_CUDA(cudaMalloc((void**)&s.d_mlp, kMlpBlob * sizeof(float)));
    PWH_CUDA(cudaMemcpyAsync(s.d_mlp, blob, kMlpBlob * sizeof(float), cudaMemcpyHostToDevice,
                             s.stream));
    PWH_CUDA(cudaStreamSynchronize(s.stream));
    s.have_mlp = true;
  });
}

pwh_status pwh_get_shells(const pwh_system* sys, int32_t* nshell, int32_t* shell_of_pw,
                          double* shell_kinetic) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && nshell, "null argument");
    const System& s = sys->s;
    *nshell = s.nshell;
    if (shell_of_pw) std::copy(s.shell_pub.begin(), s.shell_pub.end(), shell_of_pw);
    if (shell_kinetic) std::copy(s.Tshell_h.begin(), s.Tshell_h.end(), shell_kinetic);
  });
}

}  // extern "C"
