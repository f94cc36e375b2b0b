// The complex Jacobi rotation of one pivot pair, shared by the Jacobi kernels.
#pragma once
#include "common.cuh"

namespace pwh {

// Rotation J = [[c, s], [-conj(s), c]] (c real) on indices (p, q) that zeroes
// the off-diagonal element apq = A_pq of the Hermitian 2 x 2 block
// [[app, apq], [conj(apq), aqq]] in J^H A J.  Identity (c = 1, s = 0) when
// apq is zero or too small to change either diagonal entry.
template <typename T>
__device__ __forceinline__ void jacobi_rotation(cx<T> apq, T app, T aqq, T& c, cx<T>& s) {
  c = (T)1;
  s = mk<T>(0, 0);
  // |A_pq| scaled against underflow: an inaccurate modulus would make the
  // rotation non-unitary when zeta is O(1) (degenerate diagonal)
  const T mx = fmax(fabs(apq.x), fabs(apq.y));
  if (!(mx > (T)0)) return;
  // unit direction of A_pq from quotients of at most 1 (no reciprocal of a
  // possibly subnormal |A_pq|), h in [1, sqrt 2]
  const T ux = apq.x / mx, uy = apq.y / mx;
  const T h = sqrt(ux * ux + uy * uy);
  const T g = mx * h;
  // an A_pq too small to change either diagonal entry is dropped without
  // rotating (the 2 x 2 update writes it as zero)
  const bool negligible = (fabs(app) + (T)100 * g == fabs(app)) &&
                          (fabs(aqq) + (T)100 * g == fabs(aqq));
  if (negligible) return;
  const T zeta = (aqq - app) / (2 * g);
  // tan of the rotation angle, the smaller root of t^2 + 2 zeta t - 1 = 0
  // (1/(2 zeta) once zeta^2 would overflow)
  const T t = fabs(zeta) > (T)1e9 ? (T)0.5 / zeta
                                  : (zeta >= 0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
  c = (T)1 / sqrt((T)1 + t * t);
  const T e = t * c / h;
  s = mk<T>(e * ux, e * uy);
}

// The same rotation from approximate reciprocals and square roots (a few
// MUFU operations instead of IEEE divisions): c^2 + |s|^2 = 1 to a few FP32
// roundings, for the FP32 stage whose basis is re-orthonormalised afterwards.
// Off-diagonal elements below 1e-30 take the exact path (no reciprocal of a
// tiny or subnormal value).
__device__ __forceinline__ void jacobi_rotation_fast(float2 apq, float app, float aqq, float& c,
                                                     float2& s) {
  const float mx = fmaxf(fabsf(apq.x), fabsf(apq.y));
  if (!(mx >= 1e-30f)) {
    jacobi_rotation<float>(apq, app, aqq, c, s);
    return;
  }
  c = 1.f;
  s = make_float2(0.f, 0.f);
  const float r = __fdividef(1.f, mx);
  const float ux = apq.x * r, uy = apq.y * r;
  const float h2 = ux * ux + uy * uy;  // in [1, 2]
  const float ih = rsqrtf(h2);
  const float g = mx * (h2 * ih);
  const bool negligible = (fabsf(app) + 100.f * g == fabsf(app)) &&
                          (fabsf(aqq) + 100.f * g == fabsf(aqq));
  if (negligible) return;
  const float zeta = (aqq - app) * (0.5f * r * ih);
  float t;
  if (fabsf(zeta) > 1e9f) {
    t = __fdividef(0.5f, zeta);
  } else {
    const float w = 1.f + zeta * zeta;
    t = __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + w * rsqrtf(w));
  }
  c = rsqrtf(1.f + t * t);
  const float e = t * c * ih;
  s = make_float2(e * ux, e * uy);
}

// The 2 x 2 block of J^H A J on rows (pk, qk) and columns (pl, ql), from the
// block a00 = A[pk][pl], a01 = A[pk][ql], a10 = A[qk][pl], a11 = A[qk][ql]
// and the rotations (ck, sk) of the row pair and (cl, sl) of the column pair.
template <typename T>
__device__ __forceinline__ void jacobi_block(cx<T> a00, cx<T> a01, cx<T> a10, cx<T> a11, T ck,
                                             cx<T> sk, T cl, cx<T> sl, cx<T>& y00, cx<T>& y01,
                                             cx<T>& y10, cx<T>& y11) {
  const cx<T> msl = mk<T>(-sl.x, sl.y);  // -conj(s_l) = J[q][p]
  // (A J) on the block: columns (pl, ql)
  const cx<T> x00 = add<T>(scl<T>(a00, cl), mul<T>(a01, msl));
  const cx<T> x01 = add<T>(mul<T>(a00, sl), scl<T>(a01, cl));
  const cx<T> x10 = add<T>(scl<T>(a10, cl), mul<T>(a11, msl));
  const cx<T> x11 = add<T>(mul<T>(a10, sl), scl<T>(a11, cl));
  // J^H (A J): row pk = c_k x0 - s_k x1, row qk = conj(s_k) x0 + c_k x1
  const cx<T> csk = mk<T>(sk.x, -sk.y);
  y00 = sub<T>(scl<T>(x00, ck), mul<T>(sk, x10));
  y01 = sub<T>(scl<T>(x01, ck), mul<T>(sk, x11));
  y10 = add<T>(mul<T>(csk, x00), scl<T>(x10, ck));
  y11 = add<T>(mul<T>(csk, x01), scl<T>(x11, ck));
}

}  // namespace pwh
