// Contiguous-axis R2C / C2R pass kernels and twiddle generators (float).
#include "kern_impl.cuh"

namespace fft3d {
typedef float R;
}
using fft3d::R;
FFT3D_DEFINE_Z(f32)
