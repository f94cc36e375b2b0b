// Double-float instances of the compile-time specialised FFT passes: the FP64
// local part of H on the FP32 pipes.
#include "df.cuh"
#include "fft_spec_impl.cuh"

namespace pwh {
template bool spec_pass<df>(SpecPass, System&, const PassArgs&);
}  // namespace pwh
