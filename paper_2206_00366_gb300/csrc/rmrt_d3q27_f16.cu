// Kernels of the d3q27 lattice with f16 storage (every moment basis,
// forced and unforced, NSE and NCDE families).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d3q27_f16(const LaunchArgs& a) { return launch_storage<LAT_D3Q27, __half>(a); }
}  // namespace rmrt
