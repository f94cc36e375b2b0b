// Block Davidson eigensolver for the lowest nb eigenpairs of H (the iterative
// diagonalisation with subspace diagonalisation of Sec. "New parallelization
// levels"; "Davidson-like algorithm [Davidson 1975]", Sec. "Dynamic
// perturbations", optical absorption).  All vectors stay on the device in the
// library's internal plane-wave order; the host only reads the nb residual
// norms and the number of accepted new directions once per iteration.
//
// Iteration (V orthonormal, HV = H V, m columns):
//   Hs = V^H HV (new columns only, then Hermitised)          GEMM + hermitize
//   (theta, c) = lowest nb eigenpairs of Hs                   device Jacobi (FP64)
//   X = V c, HX = HV c, R = HX - X theta, ||r_n||             GEMM + k_residual
//   stop when max_n ||r_n|| <= tol
//   t_n = K_n (.) r_n for unconverged n (Teter-Payne-Allan K,   k_precond
//         reference energy <x_n|T|x_n>)
//   restart V = X, HV = HX when m would exceed m_max
//   T -= V (V^H T) twice; Cholesky-QR twice with drops       GEMM + k_cholqr
//   V <- [V T], HV <- [HV, H T]                              H|psi>
// Mixed mode runs the same loop with the reduced-precision H until
// max ||r|| <= switch_tol, then restarts from the Ritz vectors with the FP64 H
// (the FP64 phase recomputes every residual in FP64).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "common.cuh"
#include "davidson.cuh"
#include "dense.cuh"
#include "gemm.cuh"

namespace pwh {

// Precision code of the 16-bit subspace products (see sgemm), and the largest
// requested residual above which the reduced phase uses them: the 16-bit
// products bound that phase's residuals at a few 1e-4.
constexpr int kR16 = 16;
constexpr double kR16Resid = 5e-3;

struct DavWs {
  DevBuf<char> vec;    // V, HV (npw x mmax each), X, HX, R, Tw (npw x nb each)
  DevBuf<char> cg;     // Jacobi-Davidson PCG: r, z, p, q (npw x nb each), scalars
  DevBuf<char> mlp;    // learned-preconditioner factors (k x nshell)
  DevBuf<char> ovt;    // S^-1/2 psi of the generalised problem (npw x nb)
  DevBuf<char> small;  // Hs, C, theta, rn, eref, t0, Wc, S, Tr, idx, kk
  DenseWs dense;
  // plane-wave space of the current solve: the full sphere in the internal
  // order, or (real bands at k = 0) the half sphere in public order with c(0)
  // stored as c(0) / sqrt 2, so that the real inner product of two bands is
  // 2 Re of their complex one over the half sphere (m2 = 2)
  int64_t n = 0;
  const double* kin = nullptr;
  const int32_t* shell = nullptr;
  bool gamma = false;
  double m2 = 1.0;
  std::vector<pwh_davidson_trace_entry> trace;  // per Rayleigh-Ritz step of the last solve
  double* h_rn = nullptr;  // pinned host mirrors
  int* h_idx = nullptr;
  ~DavWs() {
    if (vec.p) cudaFree(vec.p);
    if (cg.p) cudaFree(cg.p);
    if (mlp.p) cudaFree(mlp.p);
    if (ovt.p) cudaFree(ovt.p);
    if (small.p) cudaFree(small.p);
    if (h_rn) cudaFreeHost(h_rn);
    if (h_idx) cudaFreeHost(h_idx);
  }
};

void free_davidson_ws(DavWs* w) { delete w; }

// ----------------------------------------------------------------- kernels --
// Starting vectors of the buffer bands: pseudo-random coefficients (two
// splitmix64 draws per entry, Steele, Lea and Flood 2014, uniform in [-1, 1)
// for the real and imaginary part) damped by 1/(1 + T_G), so that they start
// mostly on low kinetic energy.  V: npw x nbuf, column-major, internal order;
// the entry g0 (G = 0 of real bands; -1 for none) is real.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void k_buffer_start(double2* __restrict__ V, int64_t npw, int nbuf,
                               const double* __restrict__ kin, uint64_t seed, int64_t g0) {
  const int64_t tot = npw * nbuf;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = t % npw;
    const uint64_t a = splitmix64(seed + 0x9e3779b97f4a7c15ull * (uint64_t)(2 * t + 1));
    const uint64_t b = splitmix64(seed + 0x9e3779b97f4a7c15ull * (uint64_t)(2 * t + 2));
    const double d = 1.0 / (1.0 + kin[g]);
    V[t] = make_double2(((double)(a >> 11) * 0x1.0p-53 * 2.0 - 1.0) * d,
                        g == g0 ? 0.0 : ((double)(b >> 11) * 0x1.0p-53 * 2.0 - 1.0) * d);
  }
}

// R = HX - X theta per band; rn[b] = ||r_b|| (squared norm times m2, the
// metric of the band storage), eref[b] = <x|T|x>/<x|x> (the band's kinetic
// energy, the reference energy of the TPA preconditioner).
__global__ void k_residual(const double2* __restrict__ X, const double2* __restrict__ HX,
                           int64_t ld, int64_t npw, const double* __restrict__ theta,
                           const double* __restrict__ kin, double2* __restrict__ R,
                           double* __restrict__ rn, double* __restrict__ eref, double m2) {
  const int b = blockIdx.x;
  const double th = theta[b];
  const double2* x = X + (size_t)b * ld;
  const double2* hx = HX + (size_t)b * ld;
  double2* r = R + (size_t)b * ld;
  double s2 = 0.0, xt = 0.0, x2 = 0.0;
  for (int64_t i = threadIdx.x; i < npw; i += blockDim.x) {
    const double2 xi = x[i];
    double2 v = make_double2(hx[i].x - th * xi.x, hx[i].y - th * xi.y);
    r[i] = v;
    s2 += v.x * v.x + v.y * v.y;
    const double a = xi.x * xi.x + xi.y * xi.y;
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
    rn[b] = sqrt(m2 * a);
    eref[b] = (d > 0 && c > 0) ? c / d : 1.0;
  }
}

// T[:, j] = K(T_G / eref) (.) R[:, idx[j]] (K = 1 when tpa == 0); with the
// learned correction, K *= exp(s[j, shell(G)]).  t0[j] = ||t_j|| (metric m2).
__global__ void k_precond(const double2* __restrict__ R, int64_t ld, int64_t npw,
                          const int* __restrict__ idx, const double* __restrict__ eref,
                          const double* __restrict__ kin, int tpa, double2* __restrict__ T,
                          int64_t ldt, double* __restrict__ t0, const float* __restrict__ sfac,
                          const int32_t* __restrict__ shell, int nshell, double m2) {
  const int j = blockIdx.x;
  const int src = idx[j];
  const double2* r = R + (size_t)src * ld;
  double2* t = T + (size_t)j * ldt;
  const double e = eref[src];
  double s2 = 0.0;
  for (int64_t i = threadIdx.x; i < npw; i += blockDim.x) {
    double k = 1.0;
    if (tpa) {
      double x = kin[i] / e;
      double p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
      k = p / (p + 16.0 * x * x * x * x);
    }
    if (sfac) k *= exp((double)sfac[(size_t)j * nshell + shell[i]]);
    double2 v = make_double2(k * r[i].x, k * r[i].y);
    t[i] = v;
    s2 += v.x * v.x + v.y * v.y;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    t0[j] = sqrt(m2 * a);
  }
}

// After a restart from Ritz vectors: Hs[0:nb, 0:nb] = diag(theta) and the kept
// Jacobi basis of that block = identity (theta is ascending).
__global__ void k_ritz_block(double2* __restrict__ Hs, int64_t ldh, double2* __restrict__ Qk,
                             const double* __restrict__ theta, int nb) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nb * nb; t += gridDim.x * blockDim.x) {
    const int i = t % nb, j = t / nb;
    Hs[(size_t)j * ldh + i] = make_double2(i == j ? theta[i] : 0.0, 0.0);
    Qk[(size_t)j * ldh + i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

__global__ void k_sqrt(double* __restrict__ a, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = sqrt(fmax(a[i], 0.0));
}

// C = 2 Re C (M x N, ld): an inner-product matrix of half-sphere bands.
__global__ void k_real2(double2* __restrict__ C, int64_t ldc, int M, int N) {
  const int64_t tot = (int64_t)M * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % M, j = t / M;
    double2* c = C + j * ldc + i;
    *c = make_double2(2.0 * c->x, 0.0);
  }
}

// V[row] = f Re V[row] in each of nb columns (the G = 0 entry of real bands).
__global__ void k_scale_row(double2* __restrict__ V, int64_t ld, int nb, int64_t row, double f) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    double2* v = V + (size_t)b * ld + row;
    *v = make_double2(f * v->x, 0.0);
  }
}

__global__ void k_copy_cols(const double2* __restrict__ src, int64_t lds, double2* __restrict__ dst,
                            int64_t ldd, int64_t npw, int k) {
  int64_t tot = npw * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % npw, j = t / npw;
    dst[j * ldd + i] = src[j * lds + i];
  }
}

__global__ void k_perm_in(const double2* __restrict__ src, int64_t lds, int64_t npw, int nb,
                          const int32_t* __restrict__ i2p, double2* __restrict__ dst, int64_t ldd) {
  int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % npw, b = t / npw;
    dst[b * ldd + i] = src[b * lds + i2p[i]];
  }
}

__global__ void k_perm_out(const double2* __restrict__ src, int64_t lds, int64_t npw, int nb,
                           const int32_t* __restrict__ i2p, double2* __restrict__ dst, int64_t ldd) {
  int64_t tot = npw * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t % npw, b = t / npw;
    dst[b * ldd + i2p[i]] = src[b * lds + i];
  }
}

// ---------------------------------------- Jacobi-Davidson correction (PCG) --
// Column j works on band idx[j].  All per-column scalars live on the device.
// r = -R[:, idx[j]], t = 0
__global__ void k_cg_init(const double2* __restrict__ R, int64_t ld, int64_t npw,
                          const int* __restrict__ idx, double2* __restrict__ r,
                          double2* __restrict__ t) {
  const int j = blockIdx.y;
  const double2* src = R + (size_t)idx[j] * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npw;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    r[(size_t)j * npw + i] = make_double2(-v.x, -v.y);
    t[(size_t)j * npw + i] = make_double2(0.0, 0.0);
  }
}
// z = K(T_G / eref[idx[j]]) (.) r  (Teter-Payne-Allan diagonal)
__global__ void k_cg_precond(const double2* __restrict__ r, int64_t npw, const int* __restrict__ idx,
                             const double* __restrict__ eref, const double* __restrict__ kin,
                             double2* __restrict__ z, const float* __restrict__ sfac,
                             const int32_t* __restrict__ shell, int nshell) {
  const int j = blockIdx.y;
  const double e = eref[idx[j]];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npw;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = kin[i] / e;
    const double p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
    double k = p / (p + 16.0 * x * x * x * x);
    if (sfac) k *= exp((double)sfac[(size_t)j * nshell + shell[i]]);
    const double2 v = r[(size_t)j * npw + i];
    z[(size_t)j * npw + i] = make_double2(k * v.x, k * v.y);
  }
}
// out[j] = m2 Re <a_j, b_j>, one 1024-thread block per column, four element
// pairs in flight a thread (fixed-order reduction)
__global__ void __launch_bounds__(1024) k_col_dot(const double2* __restrict__ a,
                                                  const double2* __restrict__ b, int64_t npw,
                                                  double* __restrict__ out, double m2) {
  const int j = blockIdx.x;
  const double2* aj = a + (size_t)j * npw;
  const double2* bj = b + (size_t)j * npw;
  double acc = 0.0;
  int64_t i = threadIdx.x;
  const int64_t st = blockDim.x;
  for (; i + 3 * st < npw; i += 4 * st) {
    double2 x[4], y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[u] = aj[i + u * st];
      y[u] = bj[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc += x[u].x * y[u].x + x[u].y * y[u].y;
  }
  for (; i < npw; i += st) {
    const double2 x = aj[i], y = bj[i];
    acc += x.x * y.x + x.y * y.y;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a2 += red[w];
    out[j] = m2 * a2;
  }
}
// q -= theta[idx[j]] p
__global__ void k_cg_shift(double2* __restrict__ q, const double2* __restrict__ p, int64_t npw,
                           const int* __restrict__ idx, const double* __restrict__ theta) {
  const int j = blockIdx.y;
  const double th = theta[idx[j]];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npw;
       i += (int64_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)j * npw + i;
    const double2 a = q[o], b = p[o];
    q[o] = make_double2(a.x - th * b.x, a.y - th * b.y);
  }
}
// alpha = rho / <p,q> (0 where <p,q> <= 0: the column stops);  t += alpha p,
// r -= alpha q
__global__ void k_cg_step(double2* __restrict__ t, double2* __restrict__ r,
                          const double2* __restrict__ p, const double2* __restrict__ q, int64_t npw,
                          const double* __restrict__ rho, const double* __restrict__ pq) {
  const int j = blockIdx.y;
  const double alpha = (pq[j] > 0.0 && rho[j] > 0.0) ? rho[j] / pq[j] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npw;
       i += (int64_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)j * npw + i;
    const double2 pv = p[o], qv = q[o];
    t[o].x += alpha * pv.x;
    t[o].y += alpha * pv.y;
    r[o].x -= alpha * qv.x;
    r[o].y -= alpha * qv.y;
  }
}
// p = z + (rho_new / rho_old) p
__global__ void k_cg_dir(double2* __restrict__ p, const double2* __restrict__ z, int64_t npw,
                         const double* __restrict__ rho_new, const double* __restrict__ rho_old) {
  const int j = blockIdx.y;
  const double beta = rho_old[j] > 0.0 ? rho_new[j] / rho_old[j] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npw;
       i += (int64_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)j * npw + i;
    const double2 zv = z[o], pv = p[o];
    p[o] = make_double2(zv.x + beta * pv.x, zv.y + beta * pv.y);
  }
}

static int grid1d(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(152 * 16, (n + 255) / 256)); }

// ------------------------------------------------------------------ solver --
struct Layout {
  double2 *V, *HV, *X, *HX, *R, *Tw;
  double2 *Hs, *Qk, *C, *Wc, *S, *Tr;
  double *theta, *rn, *eref, *t0;
  int *idx, *kk;
};

void overlap_inv_sqrt(System& s, int nb, const double2* in, int64_t ldi, double2* out,
                      int64_t ldo, int prec);  // overlap.cu

// H on k bands of the solve's space (see DavWs); with an overlap operator the
// Loewdin form S^-1/2 H S^-1/2 of the generalised problem.
static void space_apply(System& s, DavWs& w, int k, const double2* in, double2* out, int prec) {
  if (w.gamma) {
    gamma_apply(s, k, in, w.n, out, w.n, prec, true);
  } else if (s.have_overlap) {
    double2* t = (double2*)w.ovt.p;
    overlap_inv_sqrt(s, k, in, w.n, t, w.n, prec);
    apply_internal(s, k, t, w.n, out, w.n, prec);
    overlap_inv_sqrt(s, k, out, w.n, out, w.n, prec);
  } else {
    apply_internal(s, k, in, w.n, out, w.n, prec);
  }
}

// P v = v - X (X^H v) on k columns (FP32 arithmetic, FP64 storage); W: nb x k.
static void sgemm(System& s, int prec, bool conjA, int M, int N, int K, double2 alpha,
                  const double2* A, int64_t lda, const double2* B, int64_t ldb, double2 beta,
                  double2* C, int64_t ldc, cudaStream_t st);
static void project_out(System& s, const double2* X, int nb, double2* v, int k, double2* W,
                        cudaStream_t st) {
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0), mone = make_double2(-1, 0);
  const int64_t npw = s.dav->n;
  sgemm(s, kR16, true, nb, k, (int)npw, one, X, npw, v, npw, zero, W, nb, st);
  sgemm(s, kR16, false, (int)npw, k, nb, mone, X, npw, W, nb, one, v, npw, st);
}

// Approximate solution t (npw x k) of (I-XX^H)(H-theta_j)(I-XX^H) t_j = -r_j
// for the bands idx[0..k), by `iters` steps of CG preconditioned with the TPA
// diagonal (times a per-shell factor exp(s) when sfac is given), H applied in
// reduced precision.
static void jd_correction(System& s, DavWs& w, const double2* X, int nb, const double2* R,
                          const int* idx, int k, const double* theta, const double* eref,
                          int iters, int prec, double2* t, double2* Wc, int* n_apply,
                          cudaStream_t st, const float* sfac = nullptr) {
  const int64_t npw = w.n;
  ensure(w.cg, (size_t)4 * npw * k * sizeof(double2) + 8 * (size_t)k * sizeof(double) + 256);
  double2* r = (double2*)w.cg.p;
  double2* z = r + (size_t)npw * k;
  double2* p = z + (size_t)npw * k;
  double2* q = p + (size_t)npw * k;
  double* rho[2] = {(double*)(q + (size_t)npw * k), (double*)(q + (size_t)npw * k) + k};
  double* pq = rho[1] + k;
  const dim3 g2((unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (npw + 255) / 256)), k);
  k_cg_init<<<g2, 256, 0, st>>>(R, npw, npw, idx, r, t);
  PWH_LAUNCH_CHECK();
  k_cg_precond<<<g2, 256, 0, st>>>(r, npw, idx, eref, w.kin, z, sfac, w.shell, s.nshell);
  PWH_LAUNCH_CHECK();
  project_out(s, X, nb, z, k, Wc, st);
  PWH_CUDA(cudaMemcpyAsync(p, z, (size_t)npw * k * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  k_col_dot<<<k, 1024, 0, st>>>(r, z, npw, rho[0], w.m2);
  PWH_LAUNCH_CHECK();
  // one PCG step; rho[c] holds r.z of the step, rho[c ^ 1] receives the next
  auto step = [&](int c, bool last) {
    space_apply(s, w, k, p, q, prec);
    *n_apply += k;
    k_cg_shift<<<g2, 256, 0, st>>>(q, p, npw, idx, theta);
    PWH_LAUNCH_CHECK();
    project_out(s, X, nb, q, k, Wc, st);
    k_col_dot<<<k, 1024, 0, st>>>(p, q, npw, pq, w.m2);
    PWH_LAUNCH_CHECK();
    k_cg_step<<<g2, 256, 0, st>>>(t, r, p, q, npw, rho[c], pq);
    PWH_LAUNCH_CHECK();
    if (last) return;
    k_cg_precond<<<g2, 256, 0, st>>>(r, npw, idx, eref, w.kin, z, sfac, w.shell, s.nshell);
    PWH_LAUNCH_CHECK();
    project_out(s, X, nb, z, k, Wc, st);
    k_col_dot<<<k, 1024, 0, st>>>(r, z, npw, rho[c ^ 1], w.m2);
    PWH_LAUNCH_CHECK();
    k_cg_dir<<<g2, 256, 0, st>>>(p, z, npw, rho[c ^ 1], rho[c]);
    PWH_LAUNCH_CHECK();
  };
  // Steps 0 .. iters-2 are full, the last one stops after the update of t.
  // The first step runs as plain launches (it also grows every workspace
  // these shapes need); the next full steps go in pairs, one pair captured as
  // a CUDA graph and replayed (same shapes, pointers and launch configurations
  // every pair, the two rho buffers in the same roles).  Without the kernel
  // timer only; any capture failure falls back to plain launches.
  const int full = iters - 1;
  int cur = 0, done = 0;
  if (full > 0) {
    step(cur, false);
    cur ^= 1;
    ++done;
  }
  const int pairs = (full - done) / 2;
  if (pairs >= 2 && !s.timer.on) {
    const int n_apply0 = *n_apply;
    const long long launches0 = launch_counter();
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      bool threw = false;
      try {
        step(cur, false);
        step(cur ^ 1, false);
      } catch (...) {
        threw = true;
      }
      const cudaError_t e = cudaStreamEndCapture(st, &graph);
      if (threw || e != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
    }
    cudaGetLastError();  // a refused capture leaves nothing to report
    // the capture executed nothing: undo its counts, count the replays
    const long long per_pair = launch_counter() - launches0;
    note_launches(-per_pair);
    *n_apply = n_apply0;
    if (exec) {
      for (int i = 0; i < pairs; ++i) {
        PWH_CUDA(cudaGraphLaunch(exec, st));
        note_launches(per_pair);
        *n_apply += 2 * k;
      }
      done += 2 * pairs;
      cudaGraphExecDestroy(exec);
    }
    if (graph) cudaGraphDestroy(graph);
  }
  for (; done < full; ++done) {
    step(cur, false);
    cur ^= 1;
  }
  if (iters > 0) step(cur, true);
}

static Layout carve(System& s, DavWs& w, int nb, int mmax) {
  const int64_t npw = w.n;
  const size_t nvec = (size_t)npw * (2 * (size_t)mmax + 4 * (size_t)nb);
  ensure(w.vec, nvec * sizeof(double2));
  const size_t nc = 2 * (size_t)mmax * mmax + (size_t)mmax * nb + (size_t)mmax * nb + 2 * (size_t)nb * nb;
  const size_t nd = 4 * (size_t)nb;
  ensure(w.small, nc * sizeof(double2) + nd * sizeof(double) + (2 * (size_t)nb + 8) * sizeof(int) + 256);
  Layout L;
  double2* p = (double2*)w.vec.p;
  L.V = p; p += (size_t)npw * mmax;
  L.HV = p; p += (size_t)npw * mmax;
  L.X = p; p += (size_t)npw * nb;
  L.HX = p; p += (size_t)npw * nb;
  L.R = p; p += (size_t)npw * nb;
  L.Tw = p;
  double2* q = (double2*)w.small.p;
  L.Hs = q; q += (size_t)mmax * mmax;
  L.Qk = q; q += (size_t)mmax * mmax;
  L.C = q; q += (size_t)mmax * nb;
  L.Wc = q; q += (size_t)mmax * nb;
  L.S = q; q += (size_t)nb * nb;
  L.Tr = q; q += (size_t)nb * nb;
  double* d = (double*)q;
  L.theta = d; L.rn = d + nb; L.eref = d + 2 * nb; L.t0 = d + 3 * nb;
  L.idx = (int*)(d + 4 * nb);
  L.kk = L.idx + nb;
  if (!w.h_rn) {
    PWH_CUDA(cudaMallocHost((void**)&w.h_rn, 8192 * sizeof(double)));
    PWH_CUDA(cudaMallocHost((void**)&w.h_idx, 8192 * sizeof(int)));
  }
  return L;
}

// Blocks of at least this many columns take the Newton-Schulz second pass.
constexpr int kNsMinCols = 128;

// Orthonormalise T (npw x k, ld npw, in place) by two Cholesky-QR passes; the
// first also drops columns whose norm fell below drop_rel * t0.  For blocks
// of kNsMinCols columns or more the second pass is the symmetric (Loewdin)
// orthonormalisation T S^{-1/2} by Newton-Schulz when S is close enough to
// the identity (same span, orthonormal to the same precision).  Returns the
// number of surviving columns (now the first ones of T).
static void sgemm(System& s, int prec, bool conjA, int M, int N, int K, double2 alpha,
                  const double2* A, int64_t lda, const double2* B, int64_t ldb, double2 beta,
                  double2* C, int64_t ldc, cudaStream_t st);

static int cholqr2(System& s, DavWs& w, Layout& L, double2* T, int k, const double* t0,
                   double drop_rel, cudaStream_t st, int prec = PWH_FP64,
                   int prec_first = -1) {
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  const int64_t npw = w.n;
  const int p1 = prec_first < 0 ? prec : prec_first;  // first pass may be cheaper
  sgemm(s, p1, true, k, k, (int)npw, one, T, npw, T, npw, zero, L.S, k, st);
  // the first factor only has to make T Tr well conditioned (the second pass,
  // in the phase's precision, makes it orthonormal): FP32 Cholesky always;
  // T Tr stays a combination of T's columns in the GEMM's precision
  cholqr_factor(s, w.dense, L.S, k, t0, drop_rel, L.Tr, L.kk, st, true);
  sgemm(s, p1, false, (int)npw, k, k, one, T, npw, L.Tr, k, zero, L.Tw, npw, st);
  if (k >= kNsMinCols) {
    // the kept columns (the first kk of Tw) are orthonormal to the first
    // pass's rounding: the second pass as T = Tw S^{-1/2} (k x k GEMMs on the
    // whole GPU instead of a factorisation on one SM) when S is that close
    // to the identity
    PWH_CUDA(cudaMemcpyAsync(w.h_idx + 4096, L.kk, sizeof(int), cudaMemcpyDeviceToHost, st));
    PWH_CUDA(cudaStreamSynchronize(st));
    const int kk = w.h_idx[4096];
    if (kk > 0) {
      sgemm(s, prec, true, kk, kk, (int)npw, one, L.Tw, npw, L.Tw, npw, zero, L.S, kk, st);
      if (ns_inv_sqrt(s, w.dense, L.S, kk, kk, prec == PWH_FP64, L.Tr, st)) {
        sgemm(s, prec, false, (int)npw, kk, kk, one, L.Tw, npw, L.Tr, kk, zero, T, npw, st);
        return kk;
      }
    }
  }
  sgemm(s, prec, true, k, k, (int)npw, one, L.Tw, npw, L.Tw, npw, zero, L.S, k, st);
  cholqr_factor(s, w.dense, L.S, k, nullptr, 0.0, L.Tr, L.kk, st, prec != PWH_FP64);
  sgemm(s, prec, false, (int)npw, k, k, one, L.Tw, npw, L.Tr, k, zero, T, npw, st);
  PWH_CUDA(cudaMemcpyAsync(w.h_idx + 4096, L.kk, sizeof(int), cudaMemcpyDeviceToHost, st));
  PWH_CUDA(cudaStreamSynchronize(st));
  return w.h_idx[4096];
}

// Subspace GEMMs by precision code: PWH_FP64 (the FP64 phase), kR16 (the
// 16-bit sliced tensor-core product: the reduced phase while its residuals are
// far above that product's accuracy, and the projections of the
// Jacobi-Davidson inner solves) or any other value (FP32-equivalent: the
// reduced phase close to its hand-over target).  Narrow products take the
// FP32 pipe in both reduced codes.
static void sgemm(System& s, int prec, bool conjA, int M, int N, int K, double2 alpha,
                  const double2* A, int64_t lda, const double2* B, int64_t ldb, double2 beta,
                  double2* C, int64_t ldc, cudaStream_t st) {
  if (prec == PWH_FP64)
    cgemm<double>(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
  else if (prec == kR16)
    cgemm_r16(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
  else
    cgemm_f32(s, conjA, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
  // half-sphere bands: the inner products are 2 Re of the complex ones (every
  // inner-product GEMM of the solver starts from C = 0)
  if (conjA && s.dav && s.dav->gamma && M > 0 && N > 0) {
    if (beta.x != 0.0 || beta.y != 0.0)
      throw Error{PWH_ERR_STATE, "inner-product GEMM with beta != 0 on half-sphere bands"};
    k_real2<<<grid1d((int64_t)M * N), 256, 0, st>>>(C, ldc, M, N);
    PWH_LAUNCH_CHECK();
  }
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void check_err(System& s) {
  int e = 0;
  PWH_CUDA(cudaMemcpyAsync(&e, device_error_word(s), sizeof(int), cudaMemcpyDeviceToHost, s.stream));
  PWH_CUDA(cudaStreamSynchronize(s.stream));
  if (e) {
    PWH_CUDA(cudaMemsetAsync(s.d_err, 0, sizeof(int), s.stream));
    throw Error{(pwh_status)e, "a bounded device wait gave up inside the eigensolver"};
  }
}

pwh_status davidson_solve(System& s, const pwh_davidson_opts& o, double2* psi, int64_t ldpsi,
                          double* eig, pwh_davidson_stats* stats, bool gamma) {
  if (!s.dav) s.dav = new DavWs();
  DavWs& w = *s.dav;
  w.gamma = gamma;
  w.n = gamma ? (int64_t)s.gam_pub.size() : s.npw;
  w.kin = gamma ? s.d_gam_kin : s.d_kin;
  w.shell = gamma ? s.d_gam_shell : s.d_shell;
  w.m2 = gamma ? 2.0 : 1.0;
  const int64_t npw = w.n;
  // Buffer bands: the solver iterates nbt + nbuf Ritz pairs and requires the
  // tolerance only of the lowest nbt (the bands asked for); the others are
  // converged to a looser threshold.  Without them, a requested band whose
  // near-degenerate partner lies just outside the subspace converges slowly
  // (the Jacobi-Davidson correction equation then has an eigenvalue close to
  // zero on the complement of X); with them that partner is inside X.
  const int nbt = o.nb;
  const int64_t nbuf_cap[] = {(int64_t)std::max(2, (nbt + 15) / 16), 64, 1024 - (int64_t)nbt,
                              npw - nbt, 4096 / o.max_subspace_mult - (int64_t)nbt};
  const int nbuf = (int)std::max<int64_t>(0, *std::min_element(nbuf_cap, nbuf_cap + 5));
  const int nb = nbt + nbuf;
  const int mmax = o.max_subspace_mult * nb;
  Layout L = carve(s, w, nb, mmax);
  cudaStream_t st = s.stream;
  // grow every workspace the loop can need now, so that no allocation (and no
  // device-wide synchronisation) happens inside the iterations
  jacobi_reserve(w.dense, mmax, nb);
  // the largest FP64 products of the FP64 phase: subspace matrix columns
  // (up to m_max x m_max over npw), Ritz rotations (npw x nb over m_max),
  // FP64 projector products (P x nb over npw, npw x nb over P)
  oz_reserve(s, true, mmax, mmax, (int)npw);
  oz_reserve(s, false, (int)npw, nb, mmax);
  if (s.nproj > 0) {
    oz_reserve(s, true, s.nproj, nb, (int)s.npw);
    oz_reserve(s, false, (int)s.npw, nb, s.nproj);
  }
  // and of the reduced phase (FP32-equivalent products of the same shapes,
  // the FP32 nonlocal term of the reduced-precision H)
  if (o.mixed && s.nproj > 0) ensure(s.ws_vnl, (size_t)s.npw * nb * sizeof(float2));
  if (o.precond == PWH_PRECOND_MLP) ensure(w.mlp, (size_t)nb * s.nshell * sizeof(float));
  if (o.mixed) {
    x3_reserve(s, true, mmax, mmax, (int)npw);
    x3_reserve(s, false, (int)npw, nb, mmax);
  }
  if (o.mixed && o.jd_inner > 0) {
    ensure(w.cg, (size_t)4 * npw * nb * sizeof(double2) + 8 * (size_t)nb * sizeof(double) + 256);
  }
  if (s.ace_n > 0) {
    // the ACE term's products (ace_n x nb over npw, npw x nb over ace_n)
    ensure(s.ws_ace, (size_t)s.ace_n * nb * sizeof(double2));
    oz_reserve(s, true, s.ace_n, nb, (int)s.npw);
    oz_reserve(s, false, (int)s.npw, nb, s.ace_n);
    if (o.mixed) {
      x3_reserve(s, true, s.ace_n, nb, (int)s.npw);
      x3_reserve(s, false, (int)s.npw, nb, s.ace_n);
    }
  }
  if (s.have_overlap) {
    if (gamma) throw Error{PWH_ERR_ARG, "the real-band solver takes no overlap operator"};
    // S^-1/2 psi, and the projector products of the S^-1/2 applications
    ensure(w.ovt, (size_t)npw * nb * sizeof(double2));
    ensure(s.ws_ov, (size_t)2 * s.nproj * nb * sizeof(double2));
    if (o.mixed) {
      x3_reserve(s, true, s.nproj, nb, (int)npw);
      x3_reserve(s, false, (int)npw, nb, s.nproj);
    }
  }
  if (gamma) {
    // the complex full-sphere bands that carry pairs of real ones
    ensure(s.ws_psi, (size_t)s.npw * ((nb + 1) / 2) * sizeof(double2));
    ensure(s.ws_hpsi, (size_t)s.npw * ((nb + 1) / 2) * sizeof(double2));
  }
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0), mone = make_double2(-1, 0);
  const int tpa = o.precond == PWH_PRECOND_TPA ? 1 : 0;
  pwh_davidson_stats S{};
  S.switch_iter = -1;
  const double t_start = now_s();
  double t_phase = t_start;
  w.trace.clear();
  int phase_prec = o.mixed ? (s.precision == PWH_FP64 ? PWH_MIXED : s.precision) : PWH_FP64;

  auto applyH = [&](const double2* in, double2* out, int k) {
    space_apply(s, w, k, in, out, phase_prec);
    S.n_apply += k;
    if (phase_prec == PWH_FP64) S.n_apply_fp64 += k;
  };

  // starting block: public -> internal order (and the buffer bands),
  // orthonormalise, apply H
  if (gamma) {
    // half-sphere bands keep the public order; c(0) -> c(0) / sqrt 2, real
    k_copy_cols<<<grid1d(npw * nbt), 256, 0, st>>>(psi, ldpsi, L.V, npw, npw, nbt);
    PWH_LAUNCH_CHECK();
    k_scale_row<<<(nbt + 255) / 256, 256, 0, st>>>(L.V, npw, nbt, s.gam_g0, 0.7071067811865476);
    PWH_LAUNCH_CHECK();
  } else {
    k_perm_in<<<grid1d(npw * nbt), 256, 0, st>>>(psi, ldpsi, npw, nbt, s.d_int_to_pub, L.V, npw);
    PWH_LAUNCH_CHECK();
  }
  if (nbuf > 0) {
    k_buffer_start<<<grid1d(npw * nbuf), 256, 0, st>>>(L.V + (size_t)nbt * npw, npw, nbuf, w.kin,
                                                       0x9e3779b97f4a7c15ull ^ (uint64_t)nbt,
                                                       gamma ? s.gam_g0 : -1);
    PWH_LAUNCH_CHECK();
  }
  int k0 = cholqr2(s, w, L, L.V, nb, nullptr, 0.0, st);
  if (k0 < nb) throw Error{PWH_ERR_ARG, "starting bands are linearly dependent"};
  applyH(L.V, L.HV, nb);
  int m = nb;
  int hs_valid = 0;  // leading columns of Hs that match the current V, HV
  pwh_status result = PWH_ERR_NOT_CONVERGED;
  double maxr = 0.0;
  double maxr_target = 0.0;  // over the requested bands, at the last iteration
  auto restart_from_ritz = [&](bool recompute_hx) {
    k_copy_cols<<<grid1d(npw * nb), 256, 0, st>>>(L.X, npw, L.V, npw, npw, nb);
    PWH_LAUNCH_CHECK();
    if (recompute_hx) {
      // entering the FP64 phase: make the basis orthonormal to FP64 precision
      const int kx = cholqr2(s, w, L, L.V, nb, nullptr, 0.0, st, PWH_FP64);
      if (kx < nb) throw Error{PWH_ERR_NONFINITE, "Ritz vectors lost rank at the FP64 hand-over"};
      applyH(L.V, L.HV, nb);
    } else {
      k_copy_cols<<<grid1d(npw * nb), 256, 0, st>>>(L.HX, npw, L.HV, npw, npw, nb);
      PWH_LAUNCH_CHECK();
    }
    m = nb;
    hs_valid = 0;
  };
  std::vector<double> red_hist;  // requested-band residuals of the reduced phase
  for (int it = 1;; ++it) {
    // subspace-product precision of this iteration
    const int gp = phase_prec == PWH_FP64
                       ? PWH_FP64
                       : ((it == 1 || maxr_target > kR16Resid) ? kR16 : phase_prec);
    // Rayleigh-Ritz on span(V): new columns of Hs, then its lowest nb eigenpairs
    sgemm(s, gp, true, m, m - hs_valid, (int)npw, one, L.V, npw,
          L.HV + (size_t)hs_valid * npw, npw, zero, L.Hs + (size_t)hs_valid * mmax, mmax, st);
    hermitize(L.Hs, mmax, hs_valid, m, st);
    // the leading hs_valid x hs_valid block was diagonalised last time: start there
    const int warm = hs_valid;
    hs_valid = m;
    // FP64 eigenpairs in the FP64 phase; FP32 ones (from a subspace matrix
    // that is itself FP32-accurate) in the reduced-precision phase
    const bool polish = phase_prec == PWH_FP64;
    // the reduced-precision phase needs the Ritz pairs only to well below its
    // current residuals: FP32 sweeps to 1e-3 of the last largest residual
    // (relative to the largest diagonal entry), between 4e-7 and 1e-4
    const double tol32 = polish || it == 1 ? 4e-7 : std::min(1e-4, std::max(4e-7, 1e-3 * maxr_target));
    // the FP64 phase's Ritz vectors feed residuals that stop at o.tol: an
    // off-diagonal left at 1e-3 o.tol (relative to the largest diagonal
    // entry) moves a residual by about that much and a Ritz value only to
    // second order, so the FP64 sweeps stop there (between 1e-13 and 1e-11)
    const double tol64 = std::min(1e-11, std::max(1e-13, 1e-3 * o.tol));
    jacobi_eigh(s, w.dense, L.Hs, mmax, m, nb, L.theta, L.C, st, L.Qk, mmax, warm, polish, tol32,
                tol64);
    sgemm(s, gp, false, (int)npw, nb, m, one, L.V, npw, L.C, m, zero, L.X, npw, st);
    sgemm(s, gp, false, (int)npw, nb, m, one, L.HV, npw, L.C, m, zero, L.HX, npw, st);
    k_residual<<<nb, 256, 0, st>>>(L.X, L.HX, npw, npw, L.theta, w.kin, L.R, L.rn, L.eref, w.m2);
    PWH_LAUNCH_CHECK();
    PWH_CUDA(cudaMemcpyAsync(w.h_rn, L.rn, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (s.timer.on) {
      PWH_CUDA(cudaMemcpyAsync(w.h_idx + 4100, jacobi_sweeps_word(w.dense), sizeof(int),
                               cudaMemcpyDeviceToHost, st));
      PWH_CUDA(cudaMemcpyAsync(w.h_idx + 4101, jacobi32_sweeps_word(w.dense), sizeof(int),
                               cudaMemcpyDeviceToHost, st));
    }
    PWH_CUDA(cudaStreamSynchronize(st));
    check_err(s);
    if (s.timer.on) {
      // FP64 work of the eigensolve: polish sweeps x (m-1) rounds x 20 m^2
      // operations, plus the Newton-Schulz step and Q^H H Q (4 complex GEMMs)
      const double sw = w.h_idx[4100];
      if (polish) {
        s.timer.flops[KF_JACOBI] += sw * (m - 1) * 20.0 * (double)m * m + 32.0 * (double)m * m * m;
        s.timer.bytes[KF_JACOBI] += sw * (m - 1) * 3.0 * 16.0 * (double)m * m;
      }
      // FP32 stage: per round 20 m^2 operations on A (2 x 2 blocks, both
      // triangles) and 10 m^2 on Q (the block kernel above m = 512: its own
      // count per sweep); plus the warm-start transform and the
      // Newton-Schulz step (complex GEMMs of 8 m^3 each)
      const double sw32 = w.h_idx[4101];
      const int ngemm32 = (warm ? 3 : 0) + (polish ? 0 : 3);
      const double fj = m > 512 ? sw32 * jacobi32_blk_sweep_flops(m)
                                : sw32 * (m - 1) * 30.0 * (double)m * m;
      s.timer.flops[KF_JACOBI32] += fj + ngemm32 * 8.0 * (double)m * m * m;
    }
    s.timer.resolve();
    S.iters = it;
    // maxr: over every band; maxr_t: over the requested ones (the phases'
    // decisions, termination, reported residual)
    maxr = 0.0;
    double maxr_t = 0.0;
    bool finite = true;
    for (int b = 0; b < nb; ++b) {
      if (!std::isfinite(w.h_rn[b])) finite = false;
      maxr = std::max(maxr, w.h_rn[b]);
      if (b < nbt) maxr_t = std::max(maxr_t, w.h_rn[b]);
    }
    maxr_target = maxr_t;
    // this phase's target of band b: the requested bands to tol (FP64 phase)
    // or switch_tol (reduced phase); buffer bands to 1e-3 (at least
    // switch_tol) in the reduced phase, whose operator cannot take the top
    // of the window much further, and to 1e3 tol (at most switch_tol) in the
    // FP64 phase
    const double thr = phase_prec == PWH_FP64 ? o.tol : o.switch_tol;
    const double thr_buf = phase_prec == PWH_FP64 ? std::max(o.tol, std::min(1e3 * o.tol, o.switch_tol))
                                                  : std::max(o.switch_tol, 1e-3);
    auto above = [&](int b) { return w.h_rn[b] > (b < nbt ? thr : thr_buf); };
    {
      int n_above = 0;
      for (int b = 0; b < nb; ++b) n_above += above(b);
      w.trace.push_back({it, phase_prec == PWH_FP64 ? 1 : 0, m, n_above, maxr_t, now_s() - t_start});
    }
    if (!finite) {
      result = PWH_ERR_NONFINITE;
      break;
    }
    // the hand-over waits for the requested bands only: buffer bands still
    // above their reduced-phase target are carried into the FP64 phase, whose
    // Jacobi-Davidson steps converge them anyway (waiting for them cost the
    // 512-band solve three reduced iterations at the reduced phase's floor).
    // A reduced phase that stopped improving (its arithmetic's floor above
    // switch_tol) hands over as well: the best of its last four requested-band
    // residuals not 0.8 of the best of the four before
    bool stalled = false;
    if (phase_prec != PWH_FP64) {
      red_hist.push_back(maxr_t);
      const size_t h = red_hist.size();
      if (h >= 8) {
        const double a = *std::min_element(red_hist.end() - 4, red_hist.end());
        const double b = *std::min_element(red_hist.end() - 8, red_hist.end() - 4);
        stalled = a > 0.8 * b;
      }
    }
    if (phase_prec != PWH_FP64 && (maxr_t <= o.switch_tol || stalled)) {
      // hand over to FP64: restart from the Ritz vectors with the FP64 operator
      const double t = now_s();
      S.t_mixed_s = t - t_phase;
      t_phase = t;
      S.switch_iter = it;
      phase_prec = PWH_FP64;
      restart_from_ritz(true);
      continue;
    }
    if (phase_prec == PWH_FP64 && maxr_t <= o.tol) {
      result = PWH_OK;
      break;
    }
    if (it >= o.max_iter) break;
    // bands still above this phase's target get a new direction
    int k = 0;
    for (int b = 0; b < nb; ++b)
      if (above(b)) w.h_idx[k++] = b;
    PWH_CUDA(cudaMemcpyAsync(L.idx, w.h_idx, k * sizeof(int), cudaMemcpyHostToDevice, st));
    // Jacobi-Davidson steps in the FP64 phase, and in the reduced-precision
    // phase once its residuals are within 100x of the hand-over target
    const bool jd = o.mixed && o.jd_inner > 0 &&
                    (phase_prec == PWH_FP64 || maxr_t <= 100.0 * o.switch_tol);
    if (jd || m + k > mmax) {
      restart_from_ritz(false);
      if (jd) {
        // V = X: the leading block of Hs is diag(theta), its eigenbasis the identity
        k_ritz_block<<<64, 256, 0, st>>>(L.Hs, mmax, L.Qk, L.theta, nb);
        PWH_LAUNCH_CHECK();
        hs_valid = nb;
      }
    }
    double2* T = L.V + (size_t)m * npw;
    if (jd) {
      // Jacobi-Davidson step: corrections from the reduced-precision operator
      const int red = s.precision == PWH_FP64 ? PWH_MIXED : s.precision;
      jd_correction(s, w, L.X, nb, L.R, L.idx, k, L.theta, L.eref, o.jd_inner, red, T, L.Wc,
                    &S.n_apply, st);
      k_col_dot<<<k, 1024, 0, st>>>(T, T, npw, L.t0, w.m2);
      PWH_LAUNCH_CHECK();
      k_sqrt<<<1, 256, 0, st>>>(L.t0, k);
      PWH_LAUNCH_CHECK();
    } else {
      float* sfac = nullptr;
      if (o.precond == PWH_PRECOND_MLP) {
        ensure(w.mlp, (size_t)k * s.nshell * sizeof(float));
        sfac = (float*)w.mlp.p;
        mlp_factors(s, L.idx, k, L.theta, L.rn, L.eref, sfac, st);
      }
      k_precond<<<k, 256, 0, st>>>(L.R, npw, npw, L.idx, L.eref, w.kin, tpa || sfac, T, npw, L.t0,
                                   sfac, w.shell, s.nshell, w.m2);
      PWH_LAUNCH_CHECK();
    }
    // project twice; with Jacobi-Davidson corrections (already orthogonal to X
    // in reduced precision) the first pass runs in FP32 arithmetic and the
    // second, in the phase's precision, removes what it left.  Both
    // Cholesky-QR passes stay in the phase's precision: a reduced-precision
    // T Tr would bring back components along V that nothing removes.
    const int first = jd ? kR16 : gp;
    for (int pass = 0; pass < 2; ++pass) {
      const int pp = pass == 0 ? first : gp;
      sgemm(s, pp, true, m, k, (int)npw, one, L.V, npw, T, npw, zero, L.Wc, m, st);
      sgemm(s, pp, false, (int)npw, k, m, mone, L.V, npw, L.Wc, m, one, T, npw, st);
    }
    const int kn = cholqr2(s, w, L, T, k, L.t0, 1e-10, st, gp);
    if (kn == 0) {
      restart_from_ritz(false);
      continue;
    }
    applyH(T, L.HV + (size_t)m * npw, kn);
    m += kn;
  }
  // outputs: the requested bands' eigenvalues (host) and eigenvectors
  // (public order, caller's buffer)
  PWH_CUDA(cudaMemcpyAsync(eig, L.theta, nbt * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (gamma) {
    k_copy_cols<<<grid1d(npw * nbt), 256, 0, st>>>(L.X, npw, psi, ldpsi, npw, nbt);
    PWH_LAUNCH_CHECK();
    k_scale_row<<<(nbt + 255) / 256, 256, 0, st>>>(psi, ldpsi, nbt, s.gam_g0, 1.4142135623730951);
    PWH_LAUNCH_CHECK();
  } else if (s.have_overlap) {
    // eigenvectors of H x = e S x: x = S^-1/2 phi (S-orthonormal)
    overlap_inv_sqrt(s, nbt, L.X, npw, L.R, npw, PWH_FP64);
    k_perm_out<<<grid1d(npw * nbt), 256, 0, st>>>(L.R, npw, npw, nbt, s.d_int_to_pub, psi, ldpsi);
    PWH_LAUNCH_CHECK();
  } else {
    k_perm_out<<<grid1d(npw * nbt), 256, 0, st>>>(L.X, npw, npw, nbt, s.d_int_to_pub, psi, ldpsi);
    PWH_LAUNCH_CHECK();
  }
  PWH_CUDA(cudaStreamSynchronize(st));
  check_err(s);
  const double t_end = now_s();
  if (S.switch_iter >= 0)
    S.t_fp64_s = t_end - t_phase;
  else if (o.mixed)
    S.t_mixed_s = t_end - t_phase;
  else
    S.t_fp64_s = t_end - t_phase;
  S.t_total_s = t_end - t_start;
  S.max_resid = maxr_target;
  if (stats) *stats = S;
  return result;
}

}  // namespace pwh

using namespace pwh;

extern "C" pwh_status pwh_davidson_solve(pwh_system* sys, const pwh_davidson_opts* opts,
                                         void* psi_io, int64_t ld_psi, double* eig,
                                         pwh_davidson_stats* stats) {
  pwh_status st = PWH_OK;
  pwh_status g = guarded([&] {
    PWH_CHECK_ARG(sys && opts && psi_io && eig, "null argument");
    System& s = sys->s;
    const pwh_davidson_opts& o = *opts;
    PWH_CHECK_ARG(o.nb >= 1 && o.nb <= 1024, "nb out of range [1, 1024]");
    PWH_CHECK_ARG(o.nb <= s.npw, "nb larger than the number of plane waves");
    PWH_CHECK_ARG(o.max_subspace_mult >= 2 && (int64_t)o.max_subspace_mult * o.nb <= 4096,
                  "max_subspace_mult must be >= 2 and m_max <= 4096");
    PWH_CHECK_ARG(o.max_iter >= 1, "max_iter < 1");
    PWH_CHECK_ARG(std::isfinite(o.tol) && o.tol > 0, "tol must be > 0");
    PWH_CHECK_ARG(!o.mixed || (std::isfinite(o.switch_tol) && o.switch_tol >= o.tol),
                  "switch_tol must be >= tol");
    PWH_CHECK_ARG(o.precond == PWH_PRECOND_TPA || o.precond == PWH_PRECOND_NONE ||
                      o.precond == PWH_PRECOND_MLP,
                  "unknown preconditioner");
    PWH_CHECK_ARG(ld_psi >= s.npw, "ld_psi < npw");
    if (!s.have_v) throw Error{PWH_ERR_STATE, "pwh_set_potential has not been called"};
    if (o.precond == PWH_PRECOND_MLP && !s.have_mlp)
      throw Error{PWH_ERR_STATE, "PWH_PRECOND_MLP needs pwh_set_mlp first"};
    st = davidson_solve(s, o, (double2*)psi_io, ld_psi, eig, stats);
    if (st == PWH_ERR_NOT_CONVERGED) set_error("Davidson stopped at max_iter before tol");
    if (st == PWH_ERR_NONFINITE) set_error("non-finite residual norm");
  });
  return g != PWH_OK ? g : st;
}

extern "C" pwh_status pwh_davidson_solve_gamma(pwh_system* sys, const pwh_davidson_opts* opts,
                                               void* psi_io, int64_t ld_psi, double* eig,
                                               pwh_davidson_stats* stats) {
  pwh_status st = PWH_OK;
  pwh_status g = guarded([&] {
    PWH_CHECK_ARG(sys && opts && psi_io && eig, "null argument");
    System& s = sys->s;
    const pwh_davidson_opts& o = *opts;
    gamma_prepare(s);
    const int64_t nh = (int64_t)s.gam_pub.size();
    PWH_CHECK_ARG(o.nb >= 1 && o.nb <= 1024, "nb out of range [1, 1024]");
    PWH_CHECK_ARG(o.nb <= nh, "nb larger than the half sphere");
    PWH_CHECK_ARG(o.max_subspace_mult >= 2 && (int64_t)o.max_subspace_mult * o.nb <= 4096,
                  "max_subspace_mult must be >= 2 and m_max <= 4096");
    PWH_CHECK_ARG(o.max_iter >= 1, "max_iter < 1");
    PWH_CHECK_ARG(std::isfinite(o.tol) && o.tol > 0, "tol must be > 0");
    PWH_CHECK_ARG(!o.mixed || (std::isfinite(o.switch_tol) && o.switch_tol >= o.tol),
                  "switch_tol must be >= tol");
    PWH_CHECK_ARG(o.precond == PWH_PRECOND_TPA || o.precond == PWH_PRECOND_NONE ||
                      o.precond == PWH_PRECOND_MLP,
                  "unknown preconditioner");
    PWH_CHECK_ARG(ld_psi >= nh, "ld_psi < npw_half");
    if (!s.have_v) throw Error{PWH_ERR_STATE, "pwh_set_potential has not been called"};
    if (o.precond == PWH_PRECOND_MLP && !s.have_mlp)
      throw Error{PWH_ERR_STATE, "PWH_PRECOND_MLP needs pwh_set_mlp first"};
    st = davidson_solve(s, o, (double2*)psi_io, ld_psi, eig, stats, true);
    if (st == PWH_ERR_NOT_CONVERGED) set_error("Davidson stopped at max_iter before tol");
    if (st == PWH_ERR_NONFINITE) set_error("non-finite residual norm");
  });
  return g != PWH_OK ? g : st;
}

extern "C" pwh_status pwh_davidson_solve_host(pwh_system* sys, const pwh_davidson_opts* opts,
                                              void* psi_host, double* eig,
                                              pwh_davidson_stats* stats) {
  pwh_status st = PWH_OK;
  pwh_status g = guarded([&] {
    PWH_CHECK_ARG(sys && opts && psi_host && eig, "null argument");
    System& s = sys->s;
    PWH_CHECK_ARG(opts->nb >= 1 && opts->nb <= 1024, "nb out of range [1, 1024]");
    const size_t n = (size_t)s.npw * opts->nb;
    // the device copy of the bands lives in the library's host-transfer buffer
    ensure(s.ws_host, n * sizeof(double2));
    double2* d = (double2*)s.ws_host.p;
    PWH_CUDA(cudaMemcpyAsync(d, psi_host, n * sizeof(double2), cudaMemcpyHostToDevice, s.stream));
    st = pwh_davidson_solve(sys, opts, d, s.npw, eig, stats);
    if (st != PWH_OK && st != PWH_ERR_NOT_CONVERGED) throw Error{st, pwh_last_error()};
    PWH_CUDA(cudaMemcpyAsync(psi_host, d, n * sizeof(double2), cudaMemcpyDeviceToHost, s.stream));
    PWH_CUDA(cudaStreamSynchronize(s.stream));
  });
  return g != PWH_OK ? g : st;
}

extern "C" pwh_status pwh_get_davidson_trace(const pwh_system* sys, int32_t cap,
                                             pwh_davidson_trace_entry* out, int32_t* count) {
  return guarded([&] {
    PWH_CHECK_ARG(sys && count, "null argument");
    PWH_CHECK_ARG(cap >= 0 && (cap == 0 || out), "cap < 0 or null output with cap > 0");
    const System& s = sys->s;
    const int n = s.dav ? (int)s.dav->trace.size() : 0;
    *count = n;
    for (int i = 0; i < std::min(n, (int)cap); ++i) out[i] = s.dav->trace[i];
  });
}
