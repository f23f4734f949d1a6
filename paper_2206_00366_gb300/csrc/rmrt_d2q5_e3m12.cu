// Kernels of the d2q5 lattice with e3m12 storage (every moment basis,
// forced and unforced, NSE and NCDE families).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d2q5_e3m12(const LaunchArgs& a) { return launch_storage<LAT_D2Q5, E3M12>(a); }
}  // namespace rmrt
