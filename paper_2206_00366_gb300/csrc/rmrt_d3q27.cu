// Kernels of the d3q27 lattice (all storage types, raw and central bases).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d3q27(const LaunchArgs& a) { return launch_lattice<LAT_D3Q27>(a); }
}  // namespace rmrt
