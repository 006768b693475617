// Compile-time FFT passes and fused spreading for the mesh sizes of group 2
// (MBD_FFT_GROUP2 in fft.cuh).
#include "fft.cuh"

namespace mbd {
MBD_FFT_GROUP_TU(2)
}  // namespace mbd
