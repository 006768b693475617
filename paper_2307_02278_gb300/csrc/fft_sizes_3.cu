// Compile-time FFT passes and fused spreading for the mesh sizes of group 3
// (MBD_FFT_GROUP3 in fft.cuh).
#include "fft.cuh"

namespace mbd {
MBD_FFT_GROUP_TU(3)
}  // namespace mbd
