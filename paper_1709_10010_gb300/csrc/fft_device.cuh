// Device building blocks of the FFT passes: in-register DFTs of radix 2, 3, 4,
// 5 and the in-place mixed-radix butterfly (decimation in time for inverse
// transforms, its transpose - decimation in frequency - for forward ones).
#pragma once
#include "common.cuh"

namespace pwh {

// ---------------------------------------------------------- device FFT ------
// sin/cos of 2 pi/3, 2 pi/5, 4 pi/5 (mathematical constants)
#define PWH_S3 0.866025403784438646763723170753
#define PWH_C5A 0.309016994374947424102293417183
#define PWH_S5A 0.951056516295153572116439333379
#define PWH_C5B (-0.809016994374947424102293417183)
#define PWH_S5B 0.587785252292473129168705954639

// z * (sg * i)
template <typename T> __device__ __forceinline__ cx<T> rot(cx<T> z, T sg) {
  return mk<T>(-sg * z.y, sg * z.x);
}

// In-register DFT of length R with sign sg (+1 inverse, -1 forward).
template <typename T, int R> __device__ __forceinline__ void dft(cx<T>* a, T sg);

template <typename T> __device__ __forceinline__ void dft2(cx<T>* a) {
  cx<T> t = a[0];
  a[0] = add<T>(t, a[1]);
  a[1] = sub<T>(t, a[1]);
}
template <typename T, int R> __device__ __forceinline__ void dft(cx<T>* a, T sg) {
  if constexpr (R == 2) {
    dft2<T>(a);
  } else if constexpr (R == 3) {
    cx<T> t1 = add<T>(a[1], a[2]);
    cx<T> t2 = rot<T>(sub<T>(a[1], a[2]), sg * (T)PWH_S3);
    cx<T> m = sub<T>(a[0], scl<T>(t1, (T)0.5));
    a[0] = add<T>(a[0], t1);
    a[1] = add<T>(m, t2);
    a[2] = sub<T>(m, t2);
  } else if constexpr (R == 4) {
    cx<T> s02 = add<T>(a[0], a[2]), d02 = sub<T>(a[0], a[2]);
    cx<T> s13 = add<T>(a[1], a[3]), d13 = rot<T>(sub<T>(a[1], a[3]), sg);
    a[0] = add<T>(s02, s13);
    a[2] = sub<T>(s02, s13);
    a[1] = add<T>(d02, d13);
    a[3] = sub<T>(d02, d13);
  } else if constexpr (R == 5) {
    cx<T> b1 = add<T>(a[1], a[4]), b2 = add<T>(a[2], a[3]);
    cx<T> d1 = sub<T>(a[1], a[4]), d2 = sub<T>(a[2], a[3]);
    cx<T> a0 = a[0];
    cx<T> r1 = add<T>(a0, add<T>(scl<T>(b1, (T)PWH_C5A), scl<T>(b2, (T)PWH_C5B)));
    cx<T> r2 = add<T>(a0, add<T>(scl<T>(b1, (T)PWH_C5B), scl<T>(b2, (T)PWH_C5A)));
    cx<T> i1 = rot<T>(add<T>(scl<T>(d1, (T)PWH_S5A), scl<T>(d2, (T)PWH_S5B)), sg);
    cx<T> i2 = rot<T>(sub<T>(scl<T>(d1, (T)PWH_S5B), scl<T>(d2, (T)PWH_S5A)), sg);
    a[0] = add<T>(a0, add<T>(b1, b2));
    a[1] = add<T>(r1, i1);
    a[4] = sub<T>(r1, i1);
    a[2] = add<T>(r2, i2);
    a[3] = sub<T>(r2, i2);
  }
}

// One butterfly of radix R at stage (M, L) of an n-point transform.
// DIT: twiddle the inputs, then DFT.  DIF (the transpose): DFT, then twiddle.
template <typename T, int R, bool DIT>
__device__ __forceinline__ void butterfly(cx<T>* base, int estride, int M, int k1, int twstep,
                                          const cx<T>* tw, T sg) {
  cx<T> a[R];
#pragma unroll
  for (int q = 0; q < R; ++q) a[q] = base[q * M * estride];
  if (DIT) {
#pragma unroll
    for (int q = 1; q < R; ++q) {
      cx<T> w = tw[q * k1 * twstep];
      w.y *= sg;
      a[q] = mul<T>(a[q], w);
    }
  }
  dft<T, R>(a, sg);
  if (!DIT) {
#pragma unroll
    for (int q = 1; q < R; ++q) {
      cx<T> w = tw[q * k1 * twstep];
      w.y *= sg;
      a[q] = mul<T>(a[q], w);
    }
  }
#pragma unroll
  for (int q = 0; q < R; ++q) base[q * M * estride] = a[q];
}


// Format conversions at the edges of the FFT passes (band data is FP64 in
// HBM; the FP32 passes compute in FP32).
template <typename T> __device__ __forceinline__ cx<T> widen_from64(double2 z) {
  return mk<T>((T)z.x, (T)z.y);
}
// hpsi = kin psi + v (FP64)
template <typename T>
__device__ __forceinline__ double2 kin_plus(double k, double2 p, cx<T> v) {
  return make_double2(k * p.x + (double)v.x, k * p.y + (double)v.y);
}

}  // namespace pwh
