// Kernels of the d3q19 lattice with f16 storage (every moment basis,
// forced and unforced, NSE and NCDE families).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d3q19_f16(const LaunchArgs& a) { return launch_storage<LAT_D3Q19, __half>(a); }
}  // namespace rmrt
