// FP64 instances of the compile-time specialised FFT passes.
#include "fft_spec_impl.cuh"

namespace pwh {
template bool spec_pass<double>(SpecPass, System&, const PassArgs&);
}  // namespace pwh
