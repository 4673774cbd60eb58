// Strided-axis C2C pass kernels (double).
#include "kern_impl.cuh"

namespace fft3d {
typedef double R;
}
using fft3d::R;
FFT3D_DEFINE_COL(f64)
