// Kernels of the d2q5 lattice with f64 storage (one node per thread; the
// simplified NCDE of Eq. 4-16 is the model this axis-only lattice carries).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d2q5_f64(const LaunchArgs& a) { return launch_storage<LAT_D2Q5, double>(a); }
}  // namespace rmrt
