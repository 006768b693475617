// Compile-time FFT passes and fused spreading for the mesh sizes of group 5
// (MBD_FFT_GROUP5 in fft.cuh).
#include "fft.cuh"

namespace mbd {
MBD_FFT_GROUP_TU(5)
}  // namespace mbd
