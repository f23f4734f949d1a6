// Kernels of the d3q7 lattice with f64 storage (one node per thread; the
// simplified NCDE of Eq. 4-16 is the model this axis-only lattice carries).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d3q7_f64(const LaunchArgs& a) { return launch_storage<LAT_D3Q7, double>(a); }
}  // namespace rmrt
