// Kernels of the d3q7 lattice with e3m12 storage (every moment basis,
// forced and unforced, NSE and NCDE families).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d3q7_e3m12(const LaunchArgs& a) { return launch_storage<LAT_D3Q7, E3M12>(a); }
}  // namespace rmrt
