// Host-side parameter derivation shared by the single-domain solver and the
// batched cavities: lattice directions, weights (Sec. III), rates (Eq. 4-31,
// Eq. 4-10), the S_2 block in the Sherman-Morrison form (Eq. 5-8-1) and the
// rounded kernel parameter block.  Internal header: not part of the C ABI.
#pragma once

#include <math.h>
#include <string.h>

#include "../../include/rmrtlb.h"
#include "rmrt_device.cuh"
#include "rmrt_params.h"

namespace rmrt {
namespace host {

inline int lattice_q(int lat) {
  switch (lat) {
    case RMRTLB_D2Q9: return 9;
    case RMRTLB_D3Q19: return 19;
    case RMRTLB_D2Q5: return 5;
    case RMRTLB_D3Q7: return 7;
    default: return 27;
  }
}
inline int lattice_d(int lat) { return (lat == RMRTLB_D2Q9 || lat == RMRTLB_D2Q5) ? 2 : 3; }
inline bool axis_lattice(int lat) { return lat == RMRTLB_D2Q5 || lat == RMRTLB_D3Q7; }
inline bool simple_ncde(int kind) {
  return kind == RMRTLB_EQ_NCDE_SIMPLE_LINEAR || kind == RMRTLB_EQ_NCDE_SIMPLE_QUAD;
}
inline size_t storage_size(int st) { return st == RMRTLB_ST_F64 ? 8 : (st == RMRTLB_ST_F32 ? 4 : 2); }  // 16-bit: F16, BF16, E3M12

inline void lattice_dir(int lat, int j, int e[3]) {
  if (lat == RMRTLB_D2Q9 || lat == RMRTLB_D2Q5) {   // rD2Q5: the first 5 of rD2Q9
    e[0] = Lat<LAT_D2Q9>::EX[j]; e[1] = Lat<LAT_D2Q9>::EY[j]; e[2] = 0;
  } else {
    e[0] = Dirs27::EX[j]; e[1] = Dirs27::EY[j]; e[2] = Dirs27::EZ[j];
  }
}

// All constants of a solver, in FP64.
struct Consts {
  int lat, d, q, kind, forced, storage, central;
  int nx, ny, nz;
  size_t N;
  double c[3], cs2, dt, rho0, source;
  double w[27];
  double s0, s1[3], s2[3][3], soff[3], sfree;
  double ss[3], sb[3];                 // NSE: s_s and s_b of Eq. (4-31) per axis
  double force[3], adv[3];
  int st_shift;                        // E3M12: stored value = scaled deviation * 2^st_shift (range 8 * 2^-shift)
};

inline bool rate_ok(double s) { return s > 0.0 && s < 2.0 && isfinite(s); }

// Weights from the velocity-moment constraints (Sec. III): rD2Q9 Eq. (3-3-5),
// rD3Q27 Eq. (3-3-8) with omega_19 = c_s^6/(8 c1^2 c2^2 c3^2), rD3Q19 with
// omega_19 = 0; rD2Q5 / rD3Q7 omega_a = c_s^2 / (2 c_a^2) (Remark I);
// omega_0 = 1 - sum of the others.
inline int derive_weights(Consts& k) {
  const double cs2 = k.cs2;
  double c2[3] = {k.c[0] * k.c[0], k.c[1] * k.c[1], k.c[2] * k.c[2]};
  double wax[3] = {0, 0, 0}, wedge[3] = {0, 0, 0}, wcorner = 0;  // edge: xy, xz, yz
  if (axis_lattice(k.lat)) {
    for (int a = 0; a < 3; ++a) wax[a] = cs2 / (2.0 * c2[a]);
  } else if (k.lat == RMRTLB_D2Q9) {
    const double w5 = cs2 * cs2 / (4.0 * c2[0] * c2[1]);
    wax[0] = cs2 / (2.0 * c2[0]) - 2.0 * w5;
    wax[1] = cs2 / (2.0 * c2[1]) - 2.0 * w5;
    wedge[0] = w5;
  } else {
    wcorner = k.lat == RMRTLB_D3Q27 ? cs2 * cs2 * cs2 / (8.0 * c2[0] * c2[1] * c2[2]) : 0.0;
    wedge[0] = cs2 * cs2 / (4.0 * c2[0] * c2[1]) - 2.0 * wcorner;
    wedge[1] = cs2 * cs2 / (4.0 * c2[0] * c2[2]) - 2.0 * wcorner;
    wedge[2] = cs2 * cs2 / (4.0 * c2[1] * c2[2]) - 2.0 * wcorner;
    wax[0] = cs2 / (2.0 * c2[0]) - 2.0 * (wedge[0] + wedge[1]) - 4.0 * wcorner;
    wax[1] = cs2 / (2.0 * c2[1]) - 2.0 * (wedge[0] + wedge[2]) - 4.0 * wcorner;
    wax[2] = cs2 / (2.0 * c2[2]) - 2.0 * (wedge[1] + wedge[2]) - 4.0 * wcorner;
  }
  double rest = 1.0;
  for (int j = 1; j < k.q; ++j) {
    int e[3];
    lattice_dir(k.lat, j, e);
    const int nnz = (e[0] != 0) + (e[1] != 0) + (e[2] != 0);
    double w;
    if (nnz == 1) w = wax[e[0] ? 0 : (e[1] ? 1 : 2)];
    else if (nnz == 2) w = wedge[(e[0] && e[1]) ? 0 : (e[0] ? 1 : 2)];
    else w = wcorner;
    k.w[j] = w;
    rest -= w;
  }
  k.w[0] = rest;
  for (int j = 0; j < k.q; ++j)
    if (!(k.w[j] > 0.0)) return RMRTLB_EINVAL;
  return RMRTLB_OK;
}

// Rates: Eq. (4-31) for the NSE, S_1 from the diffusivity (Eq. 4-10) for the
// NCDE, and the dense S_2 block in the Sherman-Morrison form of Eq. (5-8-1).
inline int derive_rates(Consts& k, const rmrtlb_params& p) {
  const int d = k.d;
  const double cs2 = k.cs2, dt = k.dt;
  k.sfree = p.s_free;
  if (!rate_ok(k.sfree)) return RMRTLB_EINVAL;
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) k.s2[i][j] = 0.0;
  const bool nse = k.kind == RMRTLB_EQ_NSE || k.kind == RMRTLB_EQ_NSE_HELUO;
  if (nse) {
    k.s0 = p.s0 > 0 ? p.s0 : k.sfree;
    const double s1 = p.s1 > 0 ? p.s1 : k.sfree;
    for (int a = 0; a < 3; ++a) k.s1[a] = s1;
    double ss[3], sb[3];
    for (int a = 0; a < d; ++a) {
      const double ca = k.c[a] * k.c[a] - cs2;
      ss[a] = p.s_shear[a] > 0 ? p.s_shear[a] : (p.nu > 0 ? 1.0 / (2.0 * p.nu / (ca * dt) + 0.5) : -1.0);
      sb[a] = p.s_bulk[a] > 0 ? p.s_bulk[a] : (p.nu_bulk > 0 ? 1.0 / (d * p.nu_bulk / (ca * dt) + 0.5) : -1.0);
      if (!rate_ok(ss[a]) || !rate_ok(sb[a])) return RMRTLB_EINVAL;
      k.ss[a] = ss[a];
      k.sb[a] = sb[a];
    }
    for (int i = 0; i < 3; ++i) {
      k.soff[i] = p.s_off[i] > 0 ? p.s_off[i] : (p.nu > 0 ? 1.0 / (p.nu / (cs2 * dt) + 0.5) : -1.0);
      const bool used = (d == 3) || i == 0;
      if (!used) k.soff[i] = k.sfree;
      if (!rate_ok(k.soff[i])) return RMRTLB_EINVAL;
    }
    // Sbar = A - A abar b^T A / (1 + b^T A abar), A = diag(s_s), abar = a / d,
    // a_a = (1/s_ba - 1/s_sa)(c_a^2 - c_s^2), b_b = 1/(c_b^2 - c_s^2).
    double abar[3], b[3], den = 1.0;
    for (int a = 0; a < d; ++a) {
      const double ca = k.c[a] * k.c[a] - cs2;
      abar[a] = (1.0 / sb[a] - 1.0 / ss[a]) * ca / d;
      b[a] = 1.0 / ca;
      den += b[a] * ss[a] * abar[a];
    }
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        k.s2[i][j] = (i == j ? ss[i] : 0.0) - ss[i] * abar[i] * b[j] * ss[j] / den;
  } else {
    if (!(p.diffusivity > 0)) return RMRTLB_EINVAL;
    const double tau = p.diffusivity / (cs2 * dt) + 0.5;   // K = dt c_s^2 (tau - 1/2), Eq. (4-10)
    k.s0 = k.sfree;
    for (int a = 0; a < 3; ++a) k.s1[a] = 1.0 / tau;
    if (!rate_ok(k.s1[0])) return RMRTLB_EINVAL;
    for (int i = 0; i < 3; ++i) { k.s2[i][i] = k.sfree; k.soff[i] = k.sfree; }
  }
  if (!rate_ok(k.s0) || !rate_ok(k.s1[0])) return RMRTLB_EINVAL;
  return RMRTLB_OK;
}

template <typename CT>
inline KParams<CT> to_kparams(const Consts& k) {
  KParams<CT> p;
  memset(&p, 0, sizeof(p));
  p.nx = k.nx; p.ny = k.ny; p.nz = k.nz;
  p.kind = k.kind; p.forced = k.forced; p.N = k.N;
  p.basis = k.central;
  p.rho0 = CT(k.rho0); p.cs2 = CT(k.cs2); p.dt = CT(k.dt); p.source = CT(k.source);
  p.rho0d = k.rho0;
  double c[3], c2[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = a < k.d ? k.c[a] : 1.0;
    c2[a] = c[a] * c[a];
  }
  for (int a = 0; a < 3; ++a) {
    const bool used = a < k.d;
    p.c[a] = CT(c[a]);
    p.mu2[a] = used ? CT(k.cs2 / c2[a]) : CT(0);
    p.force[a] = used ? CT(k.force[a]) : CT(0);
    p.fh[a] = used ? CT(k.force[a] / c[a]) : CT(0);
    p.adv[a] = used ? CT(k.adv[a]) : CT(0);
    p.advh[a] = used ? CT(k.adv[a] / c[a]) : CT(0);
    p.s1[a] = CT(k.s1[a]);
    p.soff[a] = CT(k.soff[a]);
    // index units: dmh_a = (1 / c_a^2) sum_b S_ab c_b^2 Xh_b
    for (int b = 0; b < 3; ++b) p.s2h[a][b] = CT(k.s2[a][b] * c2[b] / c2[a]);
  }
  if (k.lat == RMRTLB_D3Q19) {
    for (int g = 0; g < 3; ++g) {
      const int al = (g + 1) % 3, be = (g + 2) % 3;
      p.q19h[g] = CT(k.cs2 * k.cs2 * c2[g] / ((c2[g] - k.cs2) * c2[al] * c2[be]));
    }
  }
  const bool scaled = k.storage == RMRTLB_ST_F16 || k.storage == RMRTLB_ST_E3M12;
  // E3M12 values x (the scaled deviation times 2^st_shift, so that the
  // chosen range maps onto the format's [0, 8)) are carried in FP32 as
  // x * 2^(bias - 127), their code in bits 11..25 of that number: both
  // factors are part of the scale
  const int e3 = k.storage == RMRTLB_ST_E3M12 ? k.st_shift + 5 - 127 : 0;
  for (int j = 0; j < 27; ++j) {
    if (j < k.q) {
      // FP16 and E3M12 storage: power of two nearest 1/omega_j (exact to
      // apply and undo, keeps deviations out of the subnormals); BF16
      // (FP32's exponent range), FP32 and FP64 storage are unscaled
      const int e = scaled ? int(lround(-log2(k.w[j]))) : 0;
      p.sc[j] = CT(ldexp(1.0, e + e3));
      p.sinv[j] = CT(ldexp(1.0, -e - e3));
      p.wd[j] = k.w[j];
    }
  }
  p.s0 = CT(k.s0); p.sfree = CT(k.sfree);
  for (int a = 0; a < 3; ++a) {
    p.ssd[a] = k.ss[a];
    p.soffd[a] = k.soff[a];
  }
  return p;
}


// Constants of a solver from the create arguments; RMRTLB_OK or EINVAL.
inline int make_consts(Consts& k, int lattice, int nx, int ny, int nz, double dx, double dy, double dz, double dt,
                       const rmrtlb_params& params, int eq_kind, int basis, int storage) {
  memset(&k, 0, sizeof(k));
  k.lat = lattice; k.d = lattice_d(lattice); k.q = lattice_q(lattice);
  k.kind = eq_kind; k.storage = storage; k.central = basis;
  k.nx = nx; k.ny = ny; k.nz = nz; k.N = size_t(nx) * ny * nz;
  k.dt = dt;
  const double sp[3] = {dx, dy, k.d == 2 ? 1.0 : dz};
  double cmin2 = 1e300;
  for (int a = 0; a < 3; ++a) {
    k.c[a] = sp[a] / dt;
    if (a < k.d) cmin2 = fmin(cmin2, k.c[a] * k.c[a]);
  }
  // rD3Q7: c^2/3 would leave omega_0 = 0 on the standard lattice (Remark II);
  // its default is c^2/4 (weights 1/4, 1/8 there)
  k.cs2 = params.cs2 > 0 ? params.cs2 : cmin2 / (lattice == RMRTLB_D3Q7 ? 4.0 : 3.0);
  // the axis-only lattices carry only the simplified NCDE (their fourth
  // moments do not satisfy the NSE / full NCDE constraints, Remark I)
  if (axis_lattice(lattice) && !simple_ncde(eq_kind)) return RMRTLB_EINVAL;
  if (!(k.cs2 < cmin2)) return RMRTLB_EINVAL;
  k.rho0 = params.rho0;
  if (!isfinite(k.rho0)) return RMRTLB_EINVAL;
  k.source = params.source;
  for (int a = 0; a < 3; ++a) {
    k.force[a] = a < k.d ? params.force[a] : 0.0;
    k.adv[a] = a < k.d ? params.adv[a] : 0.0;
  }
  const bool nse = eq_kind == RMRTLB_EQ_NSE || eq_kind == RMRTLB_EQ_NSE_HELUO;
  k.forced = (k.source != 0.0) || (nse && (k.force[0] != 0.0 || k.force[1] != 0.0 || k.force[2] != 0.0)) ||
             simple_ncde(eq_kind);   // Eq. (4-16): G from dB/dt on every step
  if (!nse) for (int a = 0; a < 3; ++a) k.force[a] = 0.0;
  if (storage == RMRTLB_ST_E3M12) {
    // the format spans [0, 8); a range R maps onto it by 2^shift with
    // shift = floor(log2(8 / R)): the power of two at or above R
    const double R = params.storage_range > 0 ? params.storage_range : (nse ? 2.0 : 8.0);
    if (!(R >= 1.0 / 1048576.0 && R <= 128.0)) return RMRTLB_EINVAL;
    k.st_shift = int(floor(log2(8.0 / R)));
  }
  int rc = derive_weights(k);
  if (rc) return rc;
  return derive_rates(k, params);
}

}  // namespace host
}  // namespace rmrt
