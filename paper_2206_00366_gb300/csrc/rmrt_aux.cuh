// Auxiliary kernels of a solver: equilibrium initialisation, population
// set/get in canonical FP64 form, and the FP64 check (macroscopic fields,
// mass, momentum, energy, residual, stability flags).  They share the
// lattice tables, transforms and equilibrium moments of rmrt_device.cuh.
#pragma once

#include "rmrt_device.cuh"

namespace rmrt {

// fbar = f^eq(rho, u) at node x, stored where the next pull gather reads it
// (slot of x - e_j).
template <int LAT, typename ST, typename CT>
__global__ void init_eq_kernel(ST* __restrict__ f, const double* __restrict__ rho,
                               const double* __restrict__ u, const KParams<CT> p) {
  using L = Lat<LAT>;
  constexpr int D = L::D, NZ = L::NZ;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  const Nbr nb(x, y, z, p.nx, p.ny, p.nz);
  const size_t N = p.N;
  const size_t own = (size_t(z) * p.ny + y) * p.nx + x;
  const bool nse = p.kind == KIND_NSE || p.kind == KIND_NSE_HELUO;
  const CT r = CT(rho[own]);
  CT uh[3] = {CT(0), CT(0), CT(0)};
  for (int al = 0; al < D; ++al) uh[al] = nse ? CT(u[al * N + own]) / p.c[al] : p.advh[al];
  Macro<CT> mc;
  mc.dA = CT(rho[own] - double(p.rho0));
  mc.rho = r;
  eq_args(mc, r, uh, p);
  Cube<LAT, CT> q;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c)
        q.v[a][b][c] = absent<LAT>(a, b, c) ? CT(0) : meq_moment<LAT>(a, b, c, mc.dA, mc.B, mc.M, p);
  q.inverse();
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    const int dx_ = Nbr::up(ex, nb.xm, nb.x0, nb.xp);
    const int dy_ = Nbr::up(ey, nb.ym, nb.y0, nb.yp);
    const int dz_ = Nbr::up(ez, nb.zm, nb.z0, nb.zp);
    const size_t idx = (size_t(dz_) * p.ny + dy_) * p.nx + dx_;
    store_st<ST, CT>(f + j * N + idx, q.v[ex + 1][ey + 1][zi<LAT>(ez)] * p.sc[j]);
  });
}

// Canonical populations <-> storage (one plane j at a time), in FP64.
// to_storage: f[j][x - e_j] = encode(src[x]); from_storage: dst[x] = decode(f[j][x - e_j]).
template <int LAT, typename ST, typename CT>
__global__ void plane_kernel(ST* __restrict__ f, double* __restrict__ plane, int j, int to_storage,
                             const KParams<CT> p) {
  using L = Lat<LAT>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  const Nbr nb(x, y, z, p.nx, p.ny, p.nz);
  int ex = 0, ey = 0, ez = 0;
  static_for<L::Q>([&](auto J) {
    constexpr int jj = decltype(J)::value;
    constexpr int cx = L::EX[jj], cy = L::EY[jj], cz = L::EZ[jj];
    if (jj == j) { ex = cx; ey = cy; ez = cz; }
  });
  const int sx = Nbr::up(ex, nb.xm, nb.x0, nb.xp);
  const int sy = Nbr::up(ey, nb.ym, nb.y0, nb.yp);
  const int sz = Nbr::up(ez, nb.zm, nb.z0, nb.zp);
  const size_t own = (size_t(z) * p.ny + y) * p.nx + x;
  const size_t idx = (size_t(sz) * p.ny + sy) * p.nx + sx;
  ST* fj = f + size_t(j) * p.N;
  const double rest = p.wd[j] * p.rho0d;
  if (to_storage) {
    store_st<ST, CT>(fj + idx, CT((plane[own] - rest) * double(p.sc[j])));
  } else {
    plane[own] = double(load_st<ST, CT>(fj + idx)) * double(p.sinv[j]) + rest;
  }
}

// Macroscopic fields and FP64 check sums of the current populations.
// Grid-stride over the nodes (1-D grid of CHECK_THREADS-thread blocks);
// sums per block: [0] sum drho, [1..3] momentum, [4] kinetic energy,
// [5] sum |u - u_prev|^2, [6] sum |u|^2, [7] unused.  A thread takes
// several nodes of its stride at a time (two; one on the 3-D lattices in
// FP64) and issues all their population and snapshot loads before using
// any or storing the new snapshot (loads behind the snapshot stores, which
// the compiler cannot move past them, made the check four times slower).
// Per-node arithmetic is in the compute type CT, and so are a thread's
// running sums over at most CHECK_RUN nodes; each
// run is then added into FP64 sums, and threads, warps and blocks are
// reduced in FP64 in a fixed order.  (FP64 accumulation per node made the
// check FP64-pipe bound on GB300: about 20 FP64 operations per node.)  The
// residual snapshot holds u in CT (exact: u is computed in CT).
constexpr int CHECK_THREADS = 256;
constexpr int CHECK_MAX_BLOCKS = 4096;
constexpr int CHECK_RUN = 16;
// Nodes per thread at a time and resident blocks per SM, per lattice size
// (measured on the 8.4 M-node FP32 workloads: rD2Q9 two nodes and four
// blocks 0.153 ms a check, four nodes and two blocks 0.197 ms; rD3Q27 two
// and two 0.30 ms, two and four 0.59 ms).
#ifndef RMRT_CHECK_BATCH_Q9
#define RMRT_CHECK_BATCH_Q9 2
#endif
#ifndef RMRT_CHECK_MINB_Q9
#define RMRT_CHECK_MINB_Q9 4
#endif
template <int LAT, typename CT>
__host__ __device__ constexpr int check_batch() {
  return sizeof(CT) == 8 ? (Lat<LAT>::Q <= 9 ? 2 : 1) : (Lat<LAT>::Q <= 9 ? RMRT_CHECK_BATCH_Q9 : 2);
}
template <int LAT, typename CT>
__host__ __device__ constexpr int check_min_blocks() {
  return sizeof(CT) == 4 && Lat<LAT>::Q <= 9 ? RMRT_CHECK_MINB_Q9 : 2;
}

template <int LAT, typename ST, typename CT>
__global__ void __launch_bounds__(CHECK_THREADS, check_min_blocks<LAT, CT>()) check_kernel(
    const ST* __restrict__ fin, double* __restrict__ rho_out, double* __restrict__ u_out,
    double* __restrict__ uprev, int use_prev, int write_prev, double* __restrict__ partials,
    int* __restrict__ flags, const KParams<CT> p) {
  using L = Lat<LAT>;
  constexpr int D = L::D, B = check_batch<LAT, CT>();
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  CT run[7] = {CT(0), CT(0), CT(0), CT(0), CT(0), CT(0), CT(0)};
  int in_run = 0;
  CT* up = reinterpret_cast<CT*>(uprev);
  int flag = 0;
  const size_t N = p.N;
  const bool nse = p.kind == KIND_NSE || p.kind == KIND_NSE_HELUO;
  // grid-stride over nodes with the coordinates advanced by carries (no
  // per-node integer division)
  const size_t G = size_t(gridDim.x) * blockDim.x;
  const size_t n0 = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int gx = int(G % p.nx), gy = int((G / p.nx) % p.ny), gz = int(G / (size_t(p.nx) * p.ny));
  int x = int(n0 % p.nx), y = int((n0 / p.nx) % p.ny), z = int(n0 / (size_t(p.nx) * p.ny));
  const CT hdtc = CT(0.5) * p.dt;
  for (size_t nb0 = n0; nb0 < N; nb0 += B * G) {
    // the populations (and the residual snapshot) of up to B nodes
    // n = nb0 + b G, all loads before any use or store
    CT f[B][L::Q], uo[B][D];
    bool ok[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      ok[b] = nb0 + b * G < N;
#pragma unroll
      for (int al = 0; al < D; ++al) uo[b][al] = (ok[b] && up && use_prev) ? up[al * N + nb0 + b * G] : CT(0);
      const Nbr nb(x, y, z, p.nx, p.ny, p.nz);
      static_for<L::Q>([&](auto J) {
        constexpr int j = decltype(J)::value;
        constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
        const int sx = Nbr::up(ex, nb.xm, nb.x0, nb.xp);
        const int sy = Nbr::up(ey, nb.ym, nb.y0, nb.yp);
        const int sz = Nbr::up(ez, nb.zm, nb.z0, nb.zp);
        const size_t idx = (size_t(sz) * p.ny + sy) * p.nx + sx;
        f[b][j] = ok[b] ? load_st<ST, CT>(fin + j * N + idx) : CT(0);
      });
      x += gx;
      if (x >= p.nx) { x -= p.nx; ++y; }
      y += gy;
      if (y >= p.ny) { y -= p.ny; ++z; }
      z += gz;
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      if (!ok[b]) continue;
      const size_t n = nb0 + b * G;
      CT s0 = CT(0), s1[3] = {CT(0), CT(0), CT(0)};
      static_for<L::Q>([&](auto J) {
        constexpr int j = decltype(J)::value;
        constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
        const CT raw = f[b][j];
        if constexpr (std::is_same<ST, E3M12>::value) {
          if ((__float_as_uint(raw) & 0x7FFFFFFFu) >= E3M12_MAX_W) flag |= 8;   // saturated code
        }
        const CT dj = raw * p.sinv[j];
        s0 += dj;
        if (ex) s1[0] += CT(ex) * dj;
        if (ey) s1[1] += CT(ey) * dj;
        if (ez) s1[2] += CT(ez) * dj;
      });
      const CT drho = s0 + hdtc * p.source;
      const CT rho = p.rho0 + drho;
      CT u[3] = {CT(0), CT(0), CT(0)}, jm[3] = {CT(0), CT(0), CT(0)};
      const CT inv = nse ? CT(1) / (p.kind == KIND_NSE ? rho : p.rho0) : CT(0);
      for (int al = 0; al < D; ++al) {
        jm[al] = s1[al] * p.c[al] + hdtc * p.force[al];
        u[al] = nse ? jm[al] * inv : p.adv[al];
      }
      if (!nse)
        for (int al = 0; al < D; ++al) jm[al] = rho * u[al];
      if (rho_out) rho_out[n] = double(rho);
      CT u2 = CT(0), du2 = CT(0);
      for (int al = 0; al < D; ++al) {
        if (u_out) u_out[al * N + n] = double(u[al]);
        u2 += u[al] * u[al];
        if (up) {
          const CT d = u[al] - uo[b][al];
          du2 += d * d;
          if (write_prev) up[al * N + n] = u[al];
        }
      }
      run[0] += drho;
      run[1] += jm[0];
      if constexpr (D > 1) run[2] += jm[1];
      if constexpr (D > 2) run[3] += jm[2];
      run[4] += CT(0.5) * rho * u2;
      run[5] += du2;
      run[6] += u2;
      if (!(drho == drho) || !(u2 == u2) || isinf(drho) || isinf(u2)) flag |= 1;
      if (nse && rho <= CT(0)) flag |= 2;
      if (nse && u2 >= p.cs2) flag |= 4;
    }
    in_run += B;
    if (in_run >= CHECK_RUN) {
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        acc[k] += double(run[k]);
        run[k] = CT(0);
      }
      in_run = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) acc[k] += double(run[k]);
  if (partials) {
    // warp then block reduction in FP64, fixed order (deterministic)
#pragma unroll
    for (int k = 0; k < 7; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    __shared__ double sm[CHECK_THREADS / 32][7];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 7; ++k) sm[warp][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < 7) {
      double s = 0;
      for (int w = 0; w < CHECK_THREADS / 32; ++w) s += sm[w][threadIdx.x];
      partials[size_t(blockIdx.x) * 8 + threadIdx.x] = s;
    }
  }
  if (flag && flags) atomicOr(flags, flag);
}

// Local viscous stress and strain rate of the NSE (Eqs. 4-32, 4-33), in
// FP64 from the decoded populations of each node:
//   X = sum_k c_k c_k (fbar_k - f^eq_k) + (dt/2)(u Fbar + Fbar u + c_s^2 Sbar I)
//   stress_ab = -(1 - s_ab/2) X_ab,  strain_ab = stress_ab / (2 K_mu,ab)
// with s_aa = s_sa, K_mu of Eq. (4-29a) at the local density.  The second
// moment of F vanishes, so fbar's moments serve for f's.  Output planes
// xx, yy, (zz), xy, (xz, yz).  grid (ceil(nx / bx), ny, nz).
template <int LAT, typename ST, typename CT>
__global__ void stress_kernel(const ST* __restrict__ fin, double* __restrict__ stress, double* __restrict__ strain,
                              const KParams<CT> p) {
  using L = Lat<LAT>;
  constexpr int D = L::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  const Nbr nb(x, y, z, p.nx, p.ny, p.nz);
  const size_t N = p.N;
  double s0 = 0.0, s1[3] = {0.0, 0.0, 0.0}, s2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    const int sx = Nbr::up(ex, nb.xm, nb.x0, nb.xp);
    const int sy = Nbr::up(ey, nb.ym, nb.y0, nb.yp);
    const int sz = Nbr::up(ez, nb.zm, nb.z0, nb.zp);
    const double dj = double(load_st<ST, CT>(fin + j * N + (size_t(sz) * p.ny + sy) * p.nx + sx)) * double(p.sinv[j]);
    const int e[3] = {ex, ey, ez};
    s0 += dj;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s1[a] += e[a] * dj;
#pragma unroll
      for (int b = 0; b < 3; ++b) s2[a][b] += e[a] * e[b] * dj;
    }
  });
  const double dt = double(p.dt), cs2 = double(p.cs2), rho0 = p.rho0d, src = double(p.source);
  const double rho = rho0 + s0 + 0.5 * dt * src;
  const double fc = p.kind == KIND_NSE_HELUO ? rho0 : rho;
  double u[3], F[3], c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c[a] = double(p.c[a]);
    F[a] = double(p.force[a]);
    u[a] = a < D ? (s1[a] * c[a] + 0.5 * dt * F[a]) / fc : 0.0;
  }
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  int k = 0;
  for (int q = 0; q < 6; ++q) {
    const int a = pa[q], b = pb[q];
    if (a >= D || b >= D) continue;
    // sum c c fbar (the rest state omega rho0 contributes rho0 c_s^2 delta)
    const double m2 = c[a] * c[b] * s2[a][b] + (a == b ? rho0 * cs2 : 0.0);
    const double meq = (a == b ? rho * cs2 : 0.0) + fc * u[a] * u[b];
    const double X = m2 - meq + 0.5 * dt * (u[a] * F[b] + F[a] * u[b] + (a == b ? cs2 * src : 0.0));
    const double s = a == b ? p.ssd[a] : p.soffd[a + b - 1];   // xy -> 0, xz -> 1, yz -> 2
    const double K = a == b ? 0.5 * (1.0 / s - 0.5) * rho * (c[a] * c[a] - cs2) * dt : (1.0 / s - 0.5) * rho * cs2 * dt;
    const double tau = -(1.0 - 0.5 * s) * X;
    const size_t own = (size_t(z) * p.ny + y) * p.nx + x;
    if (stress) stress[size_t(k) * N + own] = tau;
    if (strain) strain[size_t(k) * N + own] = tau / (2.0 * K);
    ++k;
  }
}

}  // namespace rmrt
