// Instantiates the kernels of one lattice for every storage type and basis
// and dispatches a LaunchArgs to them.  Included once per lattice by
// rmrt_<lattice>.cu with RMRT_LAT and RMRT_LAUNCH_NAME defined.
#pragma once

#include "rmrt_aux.cuh"
#include "rmrt_device.cuh"

namespace rmrt {

template <int LAT, typename ST, typename CT, int BASIS, bool NSE>
static void launch_basis(const LaunchArgs& a, const KParams<CT>& p, const ST* fin, ST* fout) {
  constexpr bool axis_only = Lat<LAT>::Q == 5 || Lat<LAT>::Q == 7;   // one node per thread only
  if constexpr (axis_only) {
    if (p.forced) step_kernel<LAT, ST, CT, BASIS, true, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
    else step_kernel<LAT, ST, CT, BASIS, false, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
    return;
  } else if constexpr (sizeof(ST) == 2) {
    if (a.quads) {
      if (p.forced) step_kernel_x4<LAT, ST, BASIS, true, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
      else step_kernel_x4<LAT, ST, BASIS, false, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
    } else if (a.pairs) {
      if (p.forced) step_kernel_x2<LAT, ST, CT, BASIS, true, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
      else step_kernel_x2<LAT, ST, CT, BASIS, false, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
    } else {
      if (p.forced) step_kernel<LAT, ST, CT, BASIS, true, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
      else step_kernel<LAT, ST, CT, BASIS, false, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
    }
  } else if (a.pairs) {
    if (p.forced) step_kernel_x2<LAT, ST, CT, BASIS, true, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
    else step_kernel_x2<LAT, ST, CT, BASIS, false, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
  } else {
    if (p.forced) step_kernel<LAT, ST, CT, BASIS, true, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
    else step_kernel<LAT, ST, CT, BASIS, false, NSE><<<a.grid, a.block, 0, a.stream>>>(fin, fout, p);
  }
}

// a.central carries the basis (RMRTLB_BASIS_*): raw, central, Hermite,
// central-Hermite, each a compile-time variant.
template <int LAT, typename ST, typename CT, bool NSE>
static void launch_step(const LaunchArgs& a, const KParams<CT>& p, const ST* fin, ST* fout) {
  switch (a.central) {
    case 1: launch_basis<LAT, ST, CT, 1, NSE>(a, p, fin, fout); break;
    case 2: launch_basis<LAT, ST, CT, 2, NSE>(a, p, fin, fout); break;
    case 3: launch_basis<LAT, ST, CT, 3, NSE>(a, p, fin, fout); break;
    default: launch_basis<LAT, ST, CT, 0, NSE>(a, p, fin, fout); break;
  }
}

template <int LAT, typename ST, typename CT>
static cudaError_t launch_typed(const LaunchArgs& a, const KParams<CT>& p) {
  switch (a.op) {
    case OP_STEP: {
      const ST* fin = static_cast<const ST*>(a.fin);
      ST* fout = static_cast<ST*>(a.fout);
      const bool nse = p.kind == KIND_NSE || p.kind == KIND_NSE_HELUO;
      if (nse) launch_step<LAT, ST, CT, true>(a, p, fin, fout);
      else launch_step<LAT, ST, CT, false>(a, p, fin, fout);
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
    case OP_STRESS:
      stress_kernel<LAT, ST, CT><<<a.grid, a.block, 0, a.stream>>>(static_cast<const ST*>(a.fin), a.stress, a.strain,
                                                                   p);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Storage dispatch of one lattice; the typed launchers live in one
// translation unit per (lattice, storage) so that they compile in parallel.
template <int LAT, typename ST>
cudaError_t launch_storage(const LaunchArgs& a) {
  if constexpr (std::is_same<ST, double>::value) return launch_typed<LAT, double, double>(a, *a.kp64);
  else return launch_typed<LAT, ST, float>(a, *a.kp32);
}

}  // namespace rmrt
