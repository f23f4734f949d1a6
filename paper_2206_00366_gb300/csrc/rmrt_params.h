// Parameter block passed by value to every kernel of the RMRT-LB step, and
// the launch interface between the host library and the per-lattice
// translation units.  Internal header: not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace rmrt {

enum { LAT_D2Q9 = 0, LAT_D3Q19 = 1, LAT_D3Q27 = 2, LAT_D2Q5 = 3, LAT_D3Q7 = 4 };
enum {
  KIND_NSE = 0, KIND_NSE_HELUO = 1, KIND_NCDE_LINEAR = 2, KIND_NCDE_QUAD = 3,
  KIND_NCDE_SIMPLE_LINEAR = 4, KIND_NCDE_SIMPLE_QUAD = 5   // Eq. (4-16): linear EDF, G from dB/dt
};
enum { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3, ST_E3M12 = 4 };

// Constants of one solver in the compute type CT (double for FP64 storage,
// float otherwise).  Derived once on the host in FP64 and rounded.
template <typename CT>
struct KParams {
  int nx, ny, nz;
  int kind;        // KIND_*
  int forced;      // nonzero when force or source is nonzero
  int basis;       // RMRTLB_BASIS_*: bit 0 central shift N(u), bit 1 Hermite polynomials
  size_t N;        // nodes = nx * ny * nz
  CT rho0, cs2, dt, source;
  CT c[3];                             // c_a
  CT mu2[3];                           // c_s^2 / c_a^2 (index-unit second weight moment)
  CT sc[27], sinv[27];                 // storage scale (power of two ~ 1/omega_j) and its inverse
  CT s0, s1[3], s2h[3][3], soff[3], sfree;  // rates; s2h: S_2 diagonal block in index units
  CT force[3], fh[3];                  // Fbar_a and Fbar_a / c_a
  CT adv[3], advh[3];                  // NCDE advection u_a and u_a / c_a
  CT q19h[3];                          // rD3Q19 fourth-moment term in index units
  double wd[27];                       // omega_j in FP64 (population set/get)
  double rho0d;
  double ssd[3], soffd[3];             // s_sa and s_ab (xy, xz, yz) in FP64 (local stress output)
  CT* hist;                            // simplified NCDE: B(t - dt) / c_a per node, d planes (index units)
  int hist_fresh;                      // 1: no previous B yet (dB/dt taken as 0 on this step)
  unsigned seed;                       // per-step seed of the stochastic rounding of 16-bit stores
  unsigned node_base;                  // index of node 0 in the grid the random bits are drawn over
  int plane0;                          // first plane (y in 2-D, z in 3-D) of a step launch over some planes
};

enum Op { OP_STEP = 0, OP_INIT_EQ = 1, OP_PLANE = 2, OP_CHECK = 3, OP_STRESS = 4 };

struct LaunchArgs {
  Op op;
  int storage;     // ST_*
  int central;     // basis of the relaxation, RMRTLB_BASIS_* (0 raw)
  int pairs;       // OP_STEP: two nodes per thread (nx even)
  int quads;       // OP_STEP: four nodes per thread (16-bit storage, nx % 4 == 0)
  const void* fin;
  void* fout;
  const double* rho;       // OP_INIT_EQ
  const double* u;
  double* plane;           // OP_PLANE
  int j, to_storage;
  double* rho_out;         // OP_CHECK
  double* u_out;
  double* stress;          // OP_STRESS (d(d+1)/2 planes each, either may be NULL)
  double* strain;
  double* uprev;
  int use_prev, write_prev;
  double* partials;
  int* flags;
  const KParams<double>* kp64;
  const KParams<float>* kp32;
  dim3 grid, block;
  cudaStream_t stream;
};

#define RMRT_DECLARE_LAUNCH(lat) \
  cudaError_t launch_##lat##_f64(const LaunchArgs& a); \
  cudaError_t launch_##lat##_f32(const LaunchArgs& a); \
  cudaError_t launch_##lat##_f16(const LaunchArgs& a); \
  cudaError_t launch_##lat##_bf16(const LaunchArgs& a); \
  cudaError_t launch_##lat##_e3m12(const LaunchArgs& a);
RMRT_DECLARE_LAUNCH(d2q9)
RMRT_DECLARE_LAUNCH(d3q19)
RMRT_DECLARE_LAUNCH(d3q27)
RMRT_DECLARE_LAUNCH(d2q5)
RMRT_DECLARE_LAUNCH(d3q7)
#undef RMRT_DECLARE_LAUNCH
cudaError_t launch_finalize(const double* partials, size_t nblk, double* out, cudaStream_t s);

}  // namespace rmrt
