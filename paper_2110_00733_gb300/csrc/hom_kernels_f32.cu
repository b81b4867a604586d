// FP32-field instantiation of the FFT passes and Krylov kernels.
#include "hom_passes.cuh"

namespace hom {
template struct Launch<float>;
}
