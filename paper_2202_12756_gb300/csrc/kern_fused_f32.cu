// Fused plane pass kernels (float).
#include "kern_impl.cuh"

namespace fft3d {
typedef float R;
}
using fft3d::R;
FFT3D_DEFINE_FUSED(f32)
