// Kernels of the d3q27 lattice with bf16 storage (every moment basis,
// forced and unforced, NSE and NCDE families).
#include "rmrt_launch.cuh"

namespace rmrt {
cudaError_t launch_d3q27_bf16(const LaunchArgs& a) { return launch_storage<LAT_D3Q27, __nv_bfloat16>(a); }
}  // namespace rmrt
