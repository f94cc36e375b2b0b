// Local + kinetic part of H|psi>: scatter the plane-wave sphere to z-sticks,
// inverse 3D FFT, multiply by V_LOC(r), forward 3D FFT, gather back to the
// sphere and add 1/2|k+G|^2 psi.  The kinetic term acts on the plane-wave
// coefficients and V_LOC on the real-space FFT mesh (Eq. pauli_ks, Sec. "Fully
// relativistic projector augmented-wave method"); bands are pushed through the
// FFT in batches, the single-GPU counterpart of the task-group distribution of
// V psi_i products (Sec. "New parallelization levels").
//
// Conventions: G -> r uses exp(+iG.r) unscaled; r -> G uses exp(-iG.r); the
// 1/(N1 N2 N3) of the forward transform is folded into the stored V.  The
// result is the circular convolution sum_{G'} Vt(G-G') psi_{G'} with Vt the
// grid DFT of V, exactly, for any grid V.
//
// Three passes per band batch, all in shared memory:
//   k_zinv   sticks -> inverse FFT along z               (sphere -> W[b][z][s])
//   k_plane  per (band, z-plane): inverse FFT along y on the columns that hold
//            sticks, inverse FFT along x on every row, x V(r), forward FFT
//            along x, keep the stick columns, forward FFT along y, keep the
//            stick rows                                  (W -> W, in place)
//   k_zfwd   forward FFT along z, gather to the sphere, add the kinetic term
//
// 1D transforms are in-place mixed-radix (2,3,4,5) Cooley-Tukey: inverse ones
// decimate in time from digit-reversed input (the scatter writes reversed
// positions), forward ones decimate in frequency from natural input to
// digit-reversed output (the gather reads reversed positions), so no pass needs
// a separate permutation.  Twiddles e^{2 pi i t/N} come from a host FP64 table.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <string>
#include <type_traits>

#include "common.cuh"
#include "df.cuh"
#include "fft_device.cuh"
#include "fft_spec.cuh"

namespace pwh {

// ------------------------------------------------------------ host plans ----
static void make_plan(int n, FftPlan& p, std::vector<double2>& tw, std::vector<int16_t>& perm) {
  p.n = n;
  int r = n, ns = 0;
  int rad[32];
  while (r % 4 == 0) { rad[ns++] = 4; r /= 4; }
  while (r % 2 == 0) { rad[ns++] = 2; r /= 2; }
  while (r % 3 == 0) { rad[ns++] = 3; r /= 3; }
  while (r % 5 == 0) { rad[ns++] = 5; r /= 5; }
  if (r != 1 || ns > kMaxStages) throw Error{PWH_ERR_ARG, "FFT length not 2,3,5-smooth"};
  if (ns == 0) rad[ns++] = 1;  // n == 1: identity stage
  p.nstages = ns;
  int m = 1;
  for (int s = 0; s < ns; ++s) {
    p.radix[s] = rad[s];
    p.M[s] = m;
    m *= rad[s];
    p.L[s] = m;
  }
  p.tw_off = (int)tw.size();
  for (int t = 0; t < n; ++t) {
    double a = 2.0 * M_PI * (double)t / (double)n;
    tw.push_back(make_double2(std::cos(a), std::sin(a)));
  }
  // rev(p): digits c_s of p with place values prod(r_0..r_{s-1}), recombined
  // as c_{S-1} + r_{S-1}(c_{S-2} + r_{S-2}(... + r_1 c_0)); store its inverse.
  p.perm_off = (int)perm.size();
  std::vector<int16_t> irev(n);
  for (int q = 0; q < n; ++q) {
    int rem = q, acc = 0;
    int digit[kMaxStages];
    for (int s = 0; s < ns; ++s) { digit[s] = rem % rad[s]; rem /= rad[s]; }
    acc = digit[0];
    for (int s = 1; s < ns; ++s) acc = digit[s] + rad[s] * acc;
    irev[acc] = (int16_t)q;
  }
  perm.insert(perm.end(), irev.begin(), irev.end());
}

void build_fft_plans(System& s) {
  std::vector<double2> tw;
  std::vector<int16_t> perm;
  int n[3] = {s.n1, s.n2, s.n3};
  for (int d = 0; d < 3; ++d) make_plan(n[d], s.plan[d], tw, perm);
  std::vector<float2> tw32(tw.size());
  for (size_t i = 0; i < tw.size(); ++i) tw32[i] = make_float2((float)tw[i].x, (float)tw[i].y);
  PWH_CUDA(cudaMalloc((void**)&s.d_tw64, tw.size() * sizeof(double2)));
  PWH_CUDA(cudaMalloc((void**)&s.d_tw32, tw.size() * sizeof(float2)));
  PWH_CUDA(cudaMalloc((void**)&s.d_perm, perm.size() * sizeof(int16_t)));
  PWH_CUDA(cudaMemcpy(s.d_tw64, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice));
  PWH_CUDA(cudaMemcpy(s.d_tw32, tw32.data(), tw32.size() * sizeof(float2), cudaMemcpyHostToDevice));
  // double-float pairs: hi the FP32 rounding, lo the FP32 rounding of the rest
  std::vector<float4> twdf(tw.size());
  for (size_t i = 0; i < tw.size(); ++i) {
    const float xh = (float)tw[i].x, yh = (float)tw[i].y;
    twdf[i] = make_float4(xh, (float)(tw[i].x - (double)xh), yh, (float)(tw[i].y - (double)yh));
  }
  PWH_CUDA(cudaMalloc((void**)&s.d_twdf, twdf.size() * sizeof(float4)));
  PWH_CUDA(cudaMemcpy(s.d_twdf, twdf.data(), twdf.size() * sizeof(float4), cudaMemcpyHostToDevice));
  PWH_CUDA(cudaMemcpy(s.d_perm, perm.data(), perm.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
}

// nfft independent transforms of length pl.n in shared memory: transform f
// element e lives at data[f*fstride + e*estride].  All threads of the block
// take part; ends with __syncthreads().  tw: this length's table in shared
// memory.  INV: inverse (DIT, +i sign) else forward (DIF, -i sign).
template <typename T, bool INV>
__device__ void fft_block(cx<T>* data, int nfft, int fstride, int estride, const FftPlan& pl,
                          const cx<T>* tw) {
  const T sg = INV ? (T)1 : (T)-1;
  const int n = pl.n;
  for (int ss = 0; ss < pl.nstages; ++ss) {
    const int s = INV ? ss : pl.nstages - 1 - ss;
    const int R = pl.radix[s], M = pl.M[s], L = pl.L[s];
    const int nbf = n / R;
    const int twstep = n / L;
    const int total = nfft * nbf;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int f = t / nbf, j = t - f * nbf;
      int g = j / M, k1 = j - g * M;
      cx<T>* base = data + (size_t)f * fstride + (size_t)(g * L + k1) * estride;
      switch (R) {
        case 2: butterfly<T, 2, INV>(base, estride, M, k1, twstep, tw, sg); break;
        case 3: butterfly<T, 3, INV>(base, estride, M, k1, twstep, tw, sg); break;
        case 4: butterfly<T, 4, INV>(base, estride, M, k1, twstep, tw, sg); break;
        case 5: butterfly<T, 5, INV>(base, estride, M, k1, twstep, tw, sg); break;
        default: break;  // radix 1: identity
      }
    }
    __syncthreads();
  }
}

template <typename T> struct TwT;
template <> struct TwT<double> { static const double2* get(const System& s) { return s.d_tw64; } };
template <> struct TwT<float> { static const float2* get(const System& s) { return s.d_tw32; } };
template <> struct TwT<df> { static const dfc* get(const System& s) { return (const dfc*)s.d_twdf; } };

template <typename T> __device__ __forceinline__ cx<T> from64(double2 z) {
  return widen_from64<T>(z);
}

// ---------------------------------------------------- pass 1: z inverse ----
template <typename T>
__global__ void __launch_bounds__(256) k_zinv(const double2* __restrict__ psi, int64_t ldp,
                                              const int32_t* __restrict__ stick_off,
                                              const int32_t* __restrict__ stick_of,
                                              const int16_t* __restrict__ zpos, int nsticks,
                                              FftPlan pl3, const cx<T>* __restrict__ tw_g,
                                              const int16_t* __restrict__ perm_g,
                                              cx<T>* __restrict__ W, int64_t wband,
                                              int spb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n3 = pl3.n, ld = n3 + 1;
  cx<T>* buf = (cx<T>*)smem_raw;
  cx<T>* tw = buf + spb * ld;
  int16_t* irev = (int16_t*)(tw + n3);
  const int b = blockIdx.y;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nsticks - s0);
  for (int t = threadIdx.x; t < n3; t += blockDim.x) {
    tw[t] = tw_g[pl3.tw_off + t];
    irev[t] = perm_g[pl3.perm_off + t];
  }
  for (int t = threadIdx.x; t < spb * ld; t += blockDim.x) buf[t] = mk<T>(0, 0);
  __syncthreads();
  const int i0 = stick_off[s0], i1 = stick_off[s0 + ns];
  const double2* src = psi + (size_t)b * ldp;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    int s = stick_of[i] - s0;
    buf[s * ld + irev[zpos[i]]] = from64<T>(src[i]);
  }
  __syncthreads();
  fft_block<T, true>(buf, ns, ld, 1, pl3, tw);
  cx<T>* dst = W + (size_t)b * wband;
  for (int t = threadIdx.x; t < n3 * spb; t += blockDim.x) {
    int z = t / spb, s = t - z * spb;
    if (s < ns) dst[(size_t)z * nsticks + s0 + s] = buf[s * ld + z];
  }
}

// ----------------------------------------------------- pass 2: planes ------
template <typename T>
__global__ void __launch_bounds__(512) k_plane(cx<T>* __restrict__ W, int64_t wband, int nsticks,
                                               int ncols, const int32_t* __restrict__ stick_col,
                                               const int32_t* __restrict__ stick_y,
                                               const int32_t* __restrict__ col_x,
                                               const T* __restrict__ V, FftPlan pl1, FftPlan pl2,
                                               const cx<T>* __restrict__ tw_g,
                                               const int16_t* __restrict__ perm_g, int rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = pl1.n, n2 = pl2.n;
  const int ld2 = n2 + 1, ld1 = n1 + 1;
  cx<T>* C = (cx<T>*)smem_raw;                 // ncols x ld2
  cx<T>* Rw = C + (size_t)ncols * ld2;         // rows x ld1
  cx<T>* tw1 = Rw + (size_t)rows * ld1;
  cx<T>* tw2 = tw1 + n1;
  int16_t* irev1 = (int16_t*)(tw2 + n2);
  int16_t* irev2 = irev1 + n1;
  const int z = blockIdx.x, b = blockIdx.y;
  const int n3 = gridDim.x;
  cx<T>* plane = W + (size_t)b * wband + (size_t)z * nsticks;
  for (int t = threadIdx.x; t < n1; t += blockDim.x) {
    tw1[t] = tw_g[pl1.tw_off + t];
    irev1[t] = perm_g[pl1.perm_off + t];
  }
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    tw2[t] = tw_g[pl2.tw_off + t];
    irev2[t] = perm_g[pl2.perm_off + t];
  }
  for (int t = threadIdx.x; t < ncols * ld2; t += blockDim.x) C[t] = mk<T>(0, 0);
  __syncthreads();
  for (int s = threadIdx.x; s < nsticks; s += blockDim.x)
    C[stick_col[s] * ld2 + irev2[stick_y[s]]] = plane[s];
  __syncthreads();
  fft_block<T, true>(C, ncols, ld2, 1, pl2, tw2);   // inverse along y, natural order out
  const T* Vz = V + (size_t)z * n1 * n2;
  for (int y0 = 0; y0 < n2; y0 += rows) {
    const int nr = min(rows, n2 - y0);
    for (int t = threadIdx.x; t < nr * ld1; t += blockDim.x) Rw[t] = mk<T>(0, 0);
    __syncthreads();
    for (int t = threadIdx.x; t < nr * ncols; t += blockDim.x) {
      int r = t / ncols, c = t - r * ncols;
      Rw[r * ld1 + irev1[col_x[c]]] = C[c * ld2 + y0 + r];
    }
    __syncthreads();
    fft_block<T, true>(Rw, nr, ld1, 1, pl1, tw1);   // inverse along x
    for (int t = threadIdx.x; t < nr * n1; t += blockDim.x) {
      int r = t / n1, x = t - r * n1;
      Rw[r * ld1 + x] = scl<T>(Rw[r * ld1 + x], Vz[(size_t)(y0 + r) * n1 + x]);
    }
    __syncthreads();
    fft_block<T, false>(Rw, nr, ld1, 1, pl1, tw1);  // forward along x, reversed out
    for (int t = threadIdx.x; t < nr * ncols; t += blockDim.x) {
      int r = t / ncols, c = t - r * ncols;
      C[c * ld2 + y0 + r] = Rw[r * ld1 + irev1[col_x[c]]];
    }
    __syncthreads();
  }
  fft_block<T, false>(C, ncols, ld2, 1, pl2, tw2);  // forward along y, reversed out
  for (int s = threadIdx.x; s < nsticks; s += blockDim.x)
    plane[s] = C[stick_col[s] * ld2 + irev2[stick_y[s]]];
  (void)n3;
}

// ---------------------------------------- pass 3: z forward + gather + T ----
template <typename T>
__global__ void __launch_bounds__(256) k_zfwd(const cx<T>* __restrict__ W, int64_t wband,
                                              const int32_t* __restrict__ stick_off,
                                              const int32_t* __restrict__ stick_of,
                                              const int16_t* __restrict__ zpos, int nsticks,
                                              FftPlan pl3, const cx<T>* __restrict__ tw_g,
                                              const int16_t* __restrict__ perm_g,
                                              const double* __restrict__ kin,
                                              const double2* __restrict__ psi, int64_t ldp,
                                              double2* __restrict__ hpsi, int64_t ldh, int spb,
                                              const float2* __restrict__ vnl, int64_t ldv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n3 = pl3.n, ld = n3 + 1;
  cx<T>* buf = (cx<T>*)smem_raw;
  cx<T>* tw = buf + spb * ld;
  int16_t* irev = (int16_t*)(tw + n3);
  const int b = blockIdx.y;
  const int s0 = blockIdx.x * spb;
  const int ns = min(spb, nsticks - s0);
  for (int t = threadIdx.x; t < n3; t += blockDim.x) {
    tw[t] = tw_g[pl3.tw_off + t];
    irev[t] = perm_g[pl3.perm_off + t];
  }
  const cx<T>* src = W + (size_t)b * wband;
  for (int t = threadIdx.x; t < n3 * spb; t += blockDim.x) {
    int z = t / spb, s = t - z * spb;
    if (s < ns) buf[s * ld + z] = src[(size_t)z * nsticks + s0 + s];
  }
  __syncthreads();
  fft_block<T, false>(buf, ns, ld, 1, pl3, tw);
  const int i0 = stick_off[s0], i1 = stick_off[s0 + ns];
  const double2* pb = psi + (size_t)b * ldp;
  double2* hb = hpsi + (size_t)b * ldh;
  const float2* vb = vnl ? vnl + (size_t)b * ldv : nullptr;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    int s = stick_of[i] - s0;
    cx<T> v = buf[s * ld + irev[zpos[i]]];
    double2 p = pb[i];
    double k = kin[i];
    double2 h = kin_plus<T>(k, p, v);
    if (vb) {
      const float2 u = vb[i];
      h.x += (double)u.x;
      h.y += (double)u.y;
    }
    hb[i] = h;
  }
}

// ------------------------------------------------------------ launcher ------
static int stick_block(int n3) { return n3 <= 64 ? 32 : 16; }

template <typename T>
static size_t plane_smem(const System& s, int rows) {
  return ((size_t)s.ncols * (s.n2 + 1) + (size_t)rows * (s.n1 + 1) + s.n1 + s.n2) * sizeof(cx<T>) +
         (size_t)(s.n1 + s.n2) * sizeof(int16_t);
}

template <typename T>
void local_kinetic(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi, int64_t ldh,
                   cudaStream_t st, const float2* vnl, int64_t ldv) {
  if (nb <= 0) return;
  constexpr bool kDf = std::is_same<T, df>::value;
  if constexpr (std::is_same<T, double>::value) {
    // the FP64 local part in double-float arithmetic on the FP32 pipes where
    // the box has compiled passes (48-bit significands, relative rounding of
    // about 2^-46 an operation)
    if (spec_box(s)) {
      local_kinetic<df>(s, nb, psi, ldp, hpsi, ldh, st, vnl, ldv);
      return;
    }
  }
  const int64_t wband = (int64_t)s.n3 * s.nsticks;
  // batch so that the stick buffer stays around 64 MB (L2-resident between passes)
  int64_t per = wband * (int64_t)sizeof(cx<T>);
  int batch = (int)std::max<int64_t>(1, std::min<int64_t>(nb, (64ll << 20) / std::max<int64_t>(per, 1)));
  ensure(s.ws_fft, (size_t)(batch * per));
  cx<T>* W = (cx<T>*)s.ws_fft.p;
  const cx<T>* tw = TwT<T>::get(s);
  const int spb = stick_block(s.n3);
  const size_t zsmem = ((size_t)spb * (s.n3 + 1) + s.n3) * sizeof(cx<T>) + s.n3 * sizeof(int16_t);
  // plane pass: as many rows per chunk as fit in 200 KB of shared memory
  const size_t budget = 200 * 1024;
  int rows = s.n2;
  while (rows > 1 && plane_smem<T>(s, rows) > budget) rows = (rows + 1) / 2;
  const size_t psmem = plane_smem<T>(s, rows);
  if (psmem > 227 * 1024) throw Error{PWH_ERR_ARG, "FFT plane does not fit in shared memory"};
  if constexpr (!kDf) {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
      cudaFuncSetAttribute(k_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      cudaFuncSetAttribute(k_zinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      cudaFuncSetAttribute(k_zfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
  }
  const T* V = kDf ? (const T*)s.d_vdf : sizeof(T) == 8 ? (const T*)s.d_v64 : (const T*)s.d_v32;
  const bool dp = sizeof(T) == 8;  // FP64 and double-float: the FP64 timer families
  // algorithmic work per band (nominal 5 N log2 N flops per complex transform of
  // length N; bytes each pass must move at minimum)
  auto l2 = [](int n) { return std::log2((double)n); };
  const double cz = sizeof(cx<T>), ncol = s.ncols;
  const double fz = 5.0 * s.n3 * l2(s.n3) * s.nsticks;                      // z pass
  const double fp = 2.0 * s.n3 * (ncol * 5.0 * s.n2 * l2(s.n2) + s.n2 * 5.0 * s.n1 * l2(s.n1));
  const double bw = cz * (double)s.nsticks * s.n3;                          // one W slice
  const double bv = sizeof(T) * (double)s.n1 * s.n2 * s.n3;                 // V, once per launch
  // compile-time specialised kernels for cubic boxes of the common sizes,
  // the runtime-plan kernels for every other box
  for (int b0 = 0; b0 < nb; b0 += batch) {
    int bb = std::min(batch, nb - b0);
    dim3 gz((s.nsticks + spb - 1) / spb, bb);
    const float2* vb = vnl ? vnl + (size_t)b0 * ldv : nullptr;
    const PassArgs pa{psi + (size_t)b0 * ldp, ldp, hpsi + (size_t)b0 * ldh, ldh, W, wband, spb,
                      zsmem, rows, psmem, bb, V, tw, st, vb, ldv};
    {
      TimedScope ts(s, dp ? KF_FFT_ZINV64 : KF_FFT_ZINV32, st, bb * fz, bb * (16.0 * s.npw + bw));
      if (!spec_pass<T>(SPEC_ZINV, s, pa)) {
        if constexpr (kDf) {
          throw Error{PWH_ERR_ARG, "double-float FFT passes need a compiled box size"};
        } else {
          k_zinv<T><<<gz, 256, zsmem, st>>>(psi + (size_t)b0 * ldp, ldp, s.d_stick_off, s.d_stick_of,
                                             s.d_zpos, s.nsticks, s.plan[2], tw, s.d_perm, W, wband, spb);
          PWH_LAUNCH_CHECK();
        }
      }
    }
    dim3 gp(s.n3, bb);
    {
      TimedScope ts(s, dp ? KF_FFT_PLANE64 : KF_FFT_PLANE32, st, bb * fp, bb * 2.0 * bw + bv);
      if (!spec_pass<T>(SPEC_PLANE, s, pa)) {
        if constexpr (kDf) {
          throw Error{PWH_ERR_ARG, "double-float FFT passes need a compiled box size"};
        } else {
          k_plane<T><<<gp, 512, psmem, st>>>(W, wband, s.nsticks, s.ncols, s.d_stick_col, s.d_stick_y,
                                              s.d_col_x, V, s.plan[0], s.plan[1], tw, s.d_perm, rows);
          PWH_LAUNCH_CHECK();
        }
      }
    }
    {
      TimedScope ts(s, dp ? KF_FFT_ZFWD64 : KF_FFT_ZFWD32, st, bb * fz,
                    bb * (bw + 2.0 * 16.0 * s.npw + 8.0 * s.npw + (vb ? 8.0 * s.npw : 0.0)));
      if (!spec_pass<T>(SPEC_ZFWD, s, pa)) {
        if constexpr (kDf) {
          throw Error{PWH_ERR_ARG, "double-float FFT passes need a compiled box size"};
        } else {
          k_zfwd<T><<<gz, 256, zsmem, st>>>(W, wband, s.d_stick_off, s.d_stick_of, s.d_zpos, s.nsticks,
                                             s.plan[2], tw, s.d_perm, s.d_kin, psi + (size_t)b0 * ldp,
                                             ldp, hpsi + (size_t)b0 * ldh, ldh, spb, vb, ldv);
          PWH_LAUNCH_CHECK();
        }
      }
    }
  }
}

template void local_kinetic<double>(System&, int, const double2*, int64_t, double2*, int64_t,
                                    cudaStream_t, const float2*, int64_t);
template void local_kinetic<float>(System&, int, const double2*, int64_t, double2*, int64_t,
                                   cudaStream_t, const float2*, int64_t);

// ------------------------------------------------ SCF: density, full box ----
// Density of a set of bands (FP64): per z-plane and slice of bands, the
// y-inverse FFT on the stick columns and the x-inverse FFT on every row of each
// band (the first half of k_plane), then rho[z][y][x] += occ_b |psi_b|^2
// (atomic: the slices of one plane add into the same points).  W holds the
// z-inverse-transformed sticks of the batch (k_zinv).  rho: internal layout
// [i3][i2][i1], unscaled.
__global__ void __launch_bounds__(512) k_density_plane(const double2* __restrict__ W, int64_t wband,
                                                       int nsticks, int ncols,
                                                       const int32_t* __restrict__ stick_col,
                                                       const int32_t* __restrict__ stick_y,
                                                       const int32_t* __restrict__ col_x, FftPlan pl1,
                                                       FftPlan pl2, const double2* __restrict__ tw_g,
                                                       const int16_t* __restrict__ perm_g,
                                                       const double* __restrict__ occ, int nbands,
                                                       int per_slice, double* __restrict__ rho,
                                                       int rows) {
  using T = double;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = pl1.n, n2 = pl2.n;
  const int ld2 = n2 + 1, ld1 = n1 + 1;
  cx<T>* C = (cx<T>*)smem_raw;
  cx<T>* Rw = C + (size_t)ncols * ld2;
  cx<T>* tw1 = Rw + (size_t)rows * ld1;
  cx<T>* tw2 = tw1 + n1;
  int16_t* irev1 = (int16_t*)(tw2 + n2);
  int16_t* irev2 = irev1 + n1;
  const int z = blockIdx.x;
  const int bb0 = blockIdx.y * per_slice, bb1 = min(nbands, bb0 + per_slice);
  for (int t = threadIdx.x; t < n1; t += blockDim.x) {
    tw1[t] = tw_g[pl1.tw_off + t];
    irev1[t] = perm_g[pl1.perm_off + t];
  }
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    tw2[t] = tw_g[pl2.tw_off + t];
    irev2[t] = perm_g[pl2.perm_off + t];
  }
  double* rz = rho + (size_t)z * n1 * n2;
  for (int b = bb0; b < bb1; ++b) {
    const double f = occ[b];
    const cx<T>* plane = W + (size_t)b * wband + (size_t)z * nsticks;
    __syncthreads();
    for (int t = threadIdx.x; t < ncols * ld2; t += blockDim.x) C[t] = mk<T>(0, 0);
    __syncthreads();
    for (int st = threadIdx.x; st < nsticks; st += blockDim.x)
      C[stick_col[st] * ld2 + irev2[stick_y[st]]] = plane[st];
    __syncthreads();
    fft_block<T, true>(C, ncols, ld2, 1, pl2, tw2);
    for (int y0 = 0; y0 < n2; y0 += rows) {
      const int nr = min(rows, n2 - y0);
      for (int t = threadIdx.x; t < nr * ld1; t += blockDim.x) Rw[t] = mk<T>(0, 0);
      __syncthreads();
      for (int t = threadIdx.x; t < nr * ncols; t += blockDim.x) {
        const int r = t / ncols, c = t - r * ncols;
        Rw[r * ld1 + irev1[col_x[c]]] = C[c * ld2 + y0 + r];
      }
      __syncthreads();
      fft_block<T, true>(Rw, nr, ld1, 1, pl1, tw1);
      for (int t = threadIdx.x; t < nr * n1; t += blockDim.x) {
        const int r = t / n1, x = t - r * n1;
        const cx<T> v = Rw[r * ld1 + x];
        atomicAdd(rz + (size_t)(y0 + r) * n1 + x, f * (v.x * v.x + v.y * v.y));
      }
      __syncthreads();
    }
  }
}

// 1D FFTs of the full n1 x n2 x n3 box (complex FP64, C order: i3 fastest)
// along one axis: lines of `axis` (0, 1, 2 for i1, i2, i3), `lines` of them a
// block, chosen consecutive in the fastest other index so that loads and
// stores are contiguous runs.  Forward: exp(-i), natural order in and out
// (unscaled); inverse: exp(+i), unscaled.  blockIdx.y selects the box of a
// batch, boxes bstride elements apart.
__global__ void __launch_bounds__(256) k_box_fft_axis(double2* __restrict__ box, int n1, int n2,
                                                      int n3, int axis, int inverse, FftPlan pl,
                                                      const double2* __restrict__ tw_g,
                                                      const int16_t* __restrict__ perm_g, int lines,
                                                      int64_t bstride) {
  using T = double;
  box += (int64_t)blockIdx.y * bstride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = pl.n, ld = n + 1;
  cx<T>* buf = (cx<T>*)smem_raw;
  cx<T>* tw = buf + (size_t)lines * ld;
  int16_t* irev = (int16_t*)(tw + n);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    tw[t] = tw_g[pl.tw_off + t];
    irev[t] = perm_g[pl.perm_off + t];
  }
  // the two other axes: slow (os) and fast (of) with their strides
  const int64_t s1 = (int64_t)n2 * n3, s2 = n3;
  int64_t es, ss, fs;
  int nslow, nfast;
  if (axis == 2) { es = 1; ss = s1; nslow = n1; fs = s2; nfast = n2; }
  else if (axis == 1) { es = s2; ss = s1; nslow = n1; fs = 1; nfast = n3; }
  else { es = s1; ss = s2; nslow = n2; fs = 1; nfast = n3; }
  const int64_t nlines = (int64_t)nslow * nfast;
  const int64_t l0 = (int64_t)blockIdx.x * lines;
  const int nl = (int)min((int64_t)lines, nlines - l0);
  __syncthreads();
  // element e of local line j: consecutive threads walk j first when the
  // line axis is strided (contiguous runs along the fast axis), e first else
  for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
    const int j = axis == 2 ? t / n : t % nl, e = axis == 2 ? t % n : t / nl;
    const int64_t L = l0 + j;
    const double2 v = box[(L / nfast) * ss + (L % nfast) * fs + e * es];
    buf[j * ld + (inverse ? irev[e] : e)] = v;
  }
  __syncthreads();
  if (inverse)
    fft_block<T, true>(buf, nl, ld, 1, pl, tw);
  else
    fft_block<T, false>(buf, nl, ld, 1, pl, tw);
  for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
    const int j = axis == 2 ? t / n : t % nl, e = axis == 2 ? t % n : t / nl;
    const int64_t L = l0 + j;
    box[(L / nfast) * ss + (L % nfast) * fs + e * es] = buf[j * ld + (inverse ? e : irev[e])];
  }
}

void density_accumulate(System& s, int nb, const double2* psi_int, const double* occ_dev,
                        double* rho_int) {
  using T = double;
  const int64_t wband = (int64_t)s.n3 * s.nsticks;
  const int64_t per = wband * (int64_t)sizeof(cx<T>);
  const int batch = (int)std::max<int64_t>(1, std::min<int64_t>(nb, (64ll << 20) / std::max<int64_t>(per, 1)));
  ensure(s.ws_fft, (size_t)(batch * per));
  cx<T>* W = (cx<T>*)s.ws_fft.p;
  const int spb = stick_block(s.n3);
  const size_t zsmem = ((size_t)spb * (s.n3 + 1) + s.n3) * sizeof(cx<T>) + s.n3 * sizeof(int16_t);
  int rows = s.n2;
  while (rows > 1 && plane_smem<T>(s, rows) > 100 * 1024) rows = (rows + 1) / 2;
  const size_t psmem = plane_smem<T>(s, rows);
  if (psmem > 227 * 1024) throw Error{PWH_ERR_ARG, "FFT plane does not fit in shared memory"};
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_density_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_zinv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  cudaStream_t st = s.stream;
  for (int b0 = 0; b0 < nb; b0 += batch) {
    const int bb = std::min(batch, nb - b0);
    dim3 gz((s.nsticks + spb - 1) / spb, bb);
    k_zinv<T><<<gz, 256, zsmem, st>>>(psi_int + (size_t)b0 * s.npw, s.npw, s.d_stick_off,
                                       s.d_stick_of, s.d_zpos, s.nsticks, s.plan[2], s.d_tw64,
                                       s.d_perm, W, wband, spb);
    PWH_LAUNCH_CHECK();
    // slices of bands per plane: enough blocks to fill the GPU
    const int slices = std::max(1, std::min(bb, (2 * 152 + s.n3 - 1) / s.n3));
    const int per_slice = (bb + slices - 1) / slices;
    k_density_plane<<<dim3(s.n3, (bb + per_slice - 1) / per_slice), 512, psmem, st>>>(
        W, wband, s.nsticks, s.ncols, s.d_stick_col, s.d_stick_y, s.d_col_x, s.plan[0], s.plan[1],
        s.d_tw64, s.d_perm, occ_dev + b0, bb, per_slice, rho_int, rows);
    PWH_LAUNCH_CHECK();
  }
}

void box_fft(System& s, double2* box, bool inverse, int nbox, int64_t bstride) {
  const int n[3] = {s.n1, s.n2, s.n3};
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_box_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  for (int axis = 2; axis >= 0; --axis) {
    const FftPlan& pl = s.plan[axis];
    const int64_t nlines = (int64_t)n[0] * n[1] * n[2] / n[axis];
    // lines a block: 16 (a 256-byte run of the fast axis), fewer if n is large
    int lines = 16;
    while (lines > 1 && ((size_t)lines * (pl.n + 1) + pl.n) * sizeof(double2) > 96 * 1024) lines /= 2;
    const size_t smem = ((size_t)lines * (pl.n + 1) + pl.n) * sizeof(double2) + pl.n * sizeof(int16_t);
    k_box_fft_axis<<<dim3((unsigned)((nlines + lines - 1) / lines), (unsigned)nbox), 256, smem,
                     s.stream>>>(box, s.n1, s.n2, s.n3, axis, inverse ? 1 : 0, pl, s.d_tw64, s.d_perm,
                                 lines, bstride);
    PWH_LAUNCH_CHECK();
  }
}

// ------------------------------------------- allocation-free entry point ----
// Scratch for pwh_apply_local_noalloc: the stick buffer of the FFT passes lives
// in this fixed device array instead of a cudaMalloc'ed workspace.  Every GPU
// that loads the library holds it until the process exits.
constexpr size_t kNoallocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
static void* noalloc_scratch_address() {
  static std::mutex mu;
  static void* addr[128] = {};
  int dev = -1;
  PWH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) throw Error{PWH_ERR_ARG, "device ordinal out of range"};
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    PWH_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = p;
  }
  return addr[dev];
}

static void local_kinetic_noalloc(System& s, int nb, const double2* psi, int64_t ldp, double2* hpsi,
                                  int64_t ldh) {
  using T = double;
  const int64_t wband = (int64_t)s.n3 * s.nsticks;
  const size_t per = (size_t)wband * sizeof(cx<T>);
  if (per > kNoallocScratchBytes)
    throw Error{PWH_ERR_ARG, "pwh_apply_local_noalloc: one band needs a " + std::to_string(per) +
                                 "-byte stick buffer (N3 x nsticks x 16), above the " +
                                 std::to_string(kNoallocScratchBytes) + "-byte static scratch"};
  cx<T>* W = (cx<T>*)noalloc_scratch_address();
  const int batch = (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, kNoallocScratchBytes / per));
  const cx<T>* tw = s.d_tw64;
  const int spb = stick_block(s.n3);
  const size_t zsmem = ((size_t)spb * (s.n3 + 1) + s.n3) * sizeof(cx<T>) + s.n3 * sizeof(int16_t);
  const size_t budget = 200 * 1024;
  int rows = s.n2;
  while (rows > 1 && plane_smem<T>(s, rows) > budget) rows = (rows + 1) / 2;
  const size_t psmem = plane_smem<T>(s, rows);
  if (psmem > 227 * 1024) throw Error{PWH_ERR_ARG, "FFT plane does not fit in shared memory"};
  PWH_CUDA(cudaFuncSetAttribute(k_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  PWH_CUDA(cudaFuncSetAttribute(k_zinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  PWH_CUDA(cudaFuncSetAttribute(k_zfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  cudaStream_t st = s.stream;
  for (int b0 = 0; b0 < nb; b0 += batch) {
    int bb = std::min(batch, nb - b0);
    dim3 gz((s.nsticks + spb - 1) / spb, bb);
    k_zinv<T><<<gz, 256, zsmem, st>>>(psi + (size_t)b0 * ldp, ldp, s.d_stick_off, s.d_stick_of,
                                       s.d_zpos, s.nsticks, s.plan[2], tw, s.d_perm, W, wband, spb);
    PWH_LAUNCH_CHECK();
    dim3 gp(s.n3, bb);
    k_plane<T><<<gp, 512, psmem, st>>>(W, wband, s.nsticks, s.ncols, s.d_stick_col, s.d_stick_y,
                                        s.d_col_x, s.d_v64, s.plan[0], s.plan[1], tw, s.d_perm, rows);
    PWH_LAUNCH_CHECK();
    k_zfwd<T><<<gz, 256, zsmem, st>>>(W, wband, s.d_stick_off, s.d_stick_of, s.d_zpos, s.nsticks,
                                       s.plan[2], tw, s.d_perm, s.d_kin, psi + (size_t)b0 * ldp, ldp,
                                       hpsi + (size_t)b0 * ldh, ldh, spb, nullptr, 0);
    PWH_LAUNCH_CHECK();
  }
}

}  // namespace pwh

extern "C" pwh_status pwh_apply_local_noalloc(pwh_system* sys, int32_t nb, const void* psi,
                                               int64_t ld_psi, void* hpsi, int64_t ld_hpsi) {
  using namespace pwh;
  return guarded([&] {
    PWH_CHECK_ARG(sys, "null system");
    System& s = sys->s;
    PWH_CHECK_ARG(nb >= 0, "nb < 0");
    if (nb == 0) return;
    PWH_CHECK_ARG(psi && hpsi, "null band pointer");
    PWH_CHECK_ARG(ld_psi >= s.npw && ld_hpsi >= s.npw, "leading dimension < npw");
    if (!s.have_v) throw Error{PWH_ERR_STATE, "pwh_set_potential has not been called"};
    local_kinetic_noalloc(s, nb, (const double2*)psi, ld_psi, (double2*)hpsi, ld_hpsi);
  });
}
