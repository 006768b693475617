// Compile-time FFT passes and fused spreading for the mesh sizes of group 0
// (MBD_FFT_GROUP0 in fft.cuh).
#include "fft.cuh"

namespace mbd {
MBD_FFT_GROUP_TU(0)
}  // namespace mbd
