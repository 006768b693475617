// Compile-time FFT passes and fused spreading for the mesh sizes of group 4
// (MBD_FFT_GROUP4 in fft.cuh).
#include "fft.cuh"

namespace mbd {
MBD_FFT_GROUP_TU(4)
}  // namespace mbd
