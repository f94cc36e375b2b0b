// FFT passes specialised at compile time for cubic boxes of common sizes
// (interface).  The kernels are in fft_spec_impl.cuh, instantiated once per
// arithmetic in fft_spec32.cu, fft_spec64.cu and fft_specdf.cu (double-float).
#pragma once
#include "common.cuh"

namespace pwh {

// Everything one pass over a band batch needs (the same launch geometry as the
// generic passes).  psi/hpsi already point at the batch's first band.
struct PassArgs {
  const double2* psi;
  int64_t ldp;
  double2* hpsi;
  int64_t ldh;
  void* W;
  int64_t wband;
  int spb;
  size_t zsmem;
  int rows;
  size_t psmem;
  int bb;
  const void* V;
  const void* tw;
  cudaStream_t st;
  const float2* vnl;  // FP32 nonlocal term added by the z-forward pass (or null)
  int64_t ldv;
};

enum SpecPass { SPEC_ZINV = 0, SPEC_PLANE = 1, SPEC_ZFWD = 2 };

// The compiled box edges (cubic boxes only).
#define PWH_SPEC_SIZES(X) \
  X(30) X(36) X(40) X(48) X(50) X(60) X(72) X(80) X(90) X(96) X(120) X(144)

// True when the system's box has compiled passes.
inline bool spec_box(const System& s) {
  if (s.n1 != s.n2 || s.n2 != s.n3) return false;
  switch (s.n1) {
#define PWH_SPEC_BOX(n) case n:
    PWH_SPEC_SIZES(PWH_SPEC_BOX)
#undef PWH_SPEC_BOX
      return true;
    default:
      return false;
  }
}

// Launch the specialised kernel of this pass for the system's box and return
// true, or return false (nothing launched) when the box has no specialisation:
// the box is not cubic or its edge is not one of the compiled sizes.
template <typename T> bool spec_pass(SpecPass pass, System& s, const PassArgs& a);

}  // namespace pwh
