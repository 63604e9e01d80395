// Explicit instantiation of the DCT kernels for FFT lengths 2^LM, LM in {2, 3, 4, 5, 6, 7, 8}
// (split across files so that the build compiles them in parallel).
#include "dct_kernels.cuh"

namespace tvs {
TVS_DCT_INSTANTIATE(2)
TVS_DCT_INSTANTIATE(3)
TVS_DCT_INSTANTIATE(4)
TVS_DCT_INSTANTIATE(5)
TVS_DCT_INSTANTIATE(6)
TVS_DCT_INSTANTIATE(7)
TVS_DCT_INSTANTIATE(8)
}  // namespace tvs
