// Compile-time FFT passes and fused spreading for the mesh sizes of group 1
// (MBD_FFT_GROUP1 in fft.cuh).
#include "fft.cuh"

namespace mbd {
MBD_FFT_GROUP_TU(1)
}  // namespace mbd
