// Kernels of the d3q27 lattice with e3m12 storage (every moment basis,
// forced and unforced, NSE and NCDE families).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d3q27_e3m12(const LaunchArgs& a) { return launch_storage<LAT_D3Q27, E3M12>(a); }
}  // namespace rmrt
