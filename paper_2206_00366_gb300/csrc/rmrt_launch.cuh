// Instantiates the kernels of one lattice for every storage type and basis
// and dispatches a LaunchArgs to them.  Included once per lattice by
// rmrt_<lattice>.cu with RMRT_LAT and RMRT_LAUNCH_NAME defined.
#pragma once

#include "rmrt_aux.cuh"
#include "rmrt_device.cuh"

namespace rmrt {

template <int LAT, typename ST, typename CT>
static cudaError_t launch_typed(const LaunchArgs& a, const KParams<CT>& p) {
  switch (a.op) {
    case OP_STEP: {
      const ST* fin = static_cast<const ST*>(a.fin);
      ST* fout = static_cast<ST*>(a.fout);
      if (a.pairs) {
        if (a.central) {
          if (p.forced) step_kernel_x2<LAT, ST, CT, true, true><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
          else step_kernel_x2<LAT, ST, CT, true, false><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
        } else {
          if (p.forced) step_kernel_x2<LAT, ST, CT, false, true><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
          else step_kernel_x2<LAT, ST, CT, false, false><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
        }
      } else if (a.central) {
        if (p.forced) step_kernel<LAT, ST, CT, true, true><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
        else step_kernel<LAT, ST, CT, true, false><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
      } else {
        if (p.forced) step_kernel<LAT, ST, CT, false, true><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
        else step_kernel<LAT, ST, CT, false, false><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
      }
      break;
    }
    case OP_INIT_EQ:
      init_eq_kernel<LAT, ST, CT><<<a.grid, a.block, 0, a.stream>>>(static_cast<ST*>(a.fout), a.rho, a.u, p);
      break;
    case OP_PLANE:
      plane_kernel<LAT, ST, CT><<<a.grid, a.block, 0, a.stream>>>(static_cast<ST*>(a.fout), a.plane, a.j,
                                                                  a.to_storage, p);
      break;
    case OP_CHECK:
      check_kernel<LAT, ST, CT><<<a.grid, a.block, 0, a.stream>>>(
          static_cast<const ST*>(a.fin), a.rho_out, a.u_out, a.uprev, a.use_prev, a.write_prev, a.partials,
          a.flags, p);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int LAT>
static cudaError_t launch_lattice(const LaunchArgs& a) {
  switch (a.storage) {
    case ST_F64: return launch_typed<LAT, double, double>(a, *a.kp64);
    case ST_F32: return launch_typed<LAT, float, float>(a, *a.kp32);
    case ST_F16: return launch_typed<LAT, __half, float>(a, *a.kp32);
    case ST_BF16: return launch_typed<LAT, __nv_bfloat16, float>(a, *a.kp32);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rmrt
