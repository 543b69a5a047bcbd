// FP32-state instantiation of the step kernels (compiled with fast-math
// intrinsics; the time step and time stay FP64).
#include "swe_launch.cuh"

namespace swe {
template struct Launch<float>;
}
