// Kernels of the d2q9 lattice with bf16 storage (every moment basis,
// forced and unforced, NSE and NCDE families).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d2q9_bf16(const LaunchArgs& a) { return launch_storage<LAT_D2Q9, __nv_bfloat16>(a); }
}  // namespace rmrt
