// Kernels of the d2q9 lattice (all storage types, raw and central bases).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d2q9(const LaunchArgs& a) { return launch_lattice<LAT_D2Q9>(a); }
}  // namespace rmrt
