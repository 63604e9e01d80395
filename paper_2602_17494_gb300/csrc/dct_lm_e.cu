// Explicit instantiation of the DCT kernels for FFT lengths 2^LM, LM in {13}
// (split across files so that the build compiles them in parallel).
#include "dct_kernels.cuh"

namespace tvs {
TVS_DCT_INSTANTIATE(13)
}  // namespace tvs
