// Contiguous-axis R2C / C2R pass kernels and twiddle generators (double).
#include "kern_impl.cuh"

namespace fft3d {
typedef double R;
}
using fft3d::R;
FFT3D_DEFINE_Z(f64)
