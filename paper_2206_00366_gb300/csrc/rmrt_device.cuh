// Device code of the fused RMRT-LB collide-and-stream step.
//
// One thread owns one lattice node.  The populations of a node are held as a
// 3 x 3 (x 3) cube g[ix][iy][iz], ix = e_x + 1, so that the raw-moment
// transform m = M f of Eq. (5-2) factors into one 3-point transform per
// axis (the rD2Q9 and rD3Q27 monomial bases are tensor products of
// {1, c, c^2}).  rD3Q19 uses the same cube with its eight corners held at
// zero: the eight monomials with every exponent >= 1 vanish on it, and
// zeroing them before the inverse transform keeps the corners empty.
//
// Storage holds the scaled deviation s_j = (fbar_j - omega_j rho0) * sc_j,
// sc_j the power of two nearest 1/omega_j (exact to apply and to undo);
// every moment below is a moment of delta_j = fbar_j - omega_j rho0, so the
// rest state never enters the arithmetic (m(omega rho0) = m^eq(rho0, 0, 0)).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "rmrt_params.h"

namespace rmrt {

// ------------------------------------------------------------------ lattices
// Velocity order: rD2Q9 as Eq. (3-1); rD3Q27 as Eq. (3-2) with the xz block
// read as (1,0,1), (-1,0,1), (-1,0,-1), (1,0,-1); rD3Q19 = first 19.
template <int LAT> struct Lat;
template <> struct Lat<LAT_D2Q9> {
  static constexpr int D = 2, Q = 9, NZ = 1;
  static constexpr int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  static constexpr int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  static constexpr int EZ[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};
struct Dirs27 {
  static constexpr int EX[27] = {0, 1, 0, 0, -1, 0, 0, 1, -1, -1, 1, 1, -1, -1,
                                 1, 0, 0, 0, 0, 1, 1, 1, -1, -1, -1, -1, 1};
  static constexpr int EY[27] = {0, 0, 1, 0, 0, -1, 0, 1, 1, -1, -1, 0, 0, 0,
                                 0, 1, -1, -1, 1, 1, 1, -1, 1, -1, -1, 1, -1};
  static constexpr int EZ[27] = {0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 0, 1, 1, -1,
                                 -1, 1, 1, -1, -1, 1, -1, 1, 1, -1, 1, -1, -1};
};
template <> struct Lat<LAT_D3Q27> : Dirs27 {
  static constexpr int D = 3, Q = 27, NZ = 3;
};
template <> struct Lat<LAT_D3Q19> : Dirs27 {
  static constexpr int D = 3, Q = 19, NZ = 3;
};

// compile-time loop: f(std::integral_constant<int, i>) for i = 0..N-1
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ------------------------------------------------------------------ storage
template <typename ST, typename CT> __device__ __forceinline__ CT load_st(const ST* p) {
  return static_cast<CT>(__ldg(p));
}
template <> __device__ __forceinline__ float load_st<__half, float>(const __half* p) {
  return __half2float(__ldg(p));
}
template <> __device__ __forceinline__ float load_st<__nv_bfloat16, float>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <typename ST, typename CT> __device__ __forceinline__ void store_st(ST* p, CT v) {
  *p = static_cast<ST>(v);
}
template <> __device__ __forceinline__ void store_st<__half, float>(__half* p, float v) {
  *p = __float2half_rn(v);
}
template <> __device__ __forceinline__ void store_st<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

// ------------------------------------------------------------------ node geometry
// Source node of the pull gather for direction e: x - e with periodic wrap.
struct Nbr {
  int xm, x0, xp, ym, y0, yp, zm, z0, zp;
  __device__ __forceinline__ Nbr(int x, int y, int z, int nx, int ny, int nz) {
    x0 = x; y0 = y; z0 = z;
    xm = x == 0 ? nx - 1 : x - 1; xp = x == nx - 1 ? 0 : x + 1;
    ym = y == 0 ? ny - 1 : y - 1; yp = y == ny - 1 ? 0 : y + 1;
    zm = z == 0 ? nz - 1 : z - 1; zp = z == nz - 1 ? 0 : z + 1;
  }
  // coordinate of x - e along one axis
  __device__ __forceinline__ static int up(int e, int m, int c, int p) { return e > 0 ? m : (e < 0 ? p : c); }
  // coordinate of x + e along one axis
  __device__ __forceinline__ static int dn(int e, int m, int c, int p) { return e > 0 ? p : (e < 0 ? m : c); }
};

// ------------------------------------------------------------------ 1-D transforms
// The moments are index moments mh_abc = sum_j e_jx^a e_jy^b e_jz^c f_j; the
// physical raw moments of Eq. (5-2) are m_abc = c_x^a c_y^b c_z^c mh_abc.
// Every constant that meets a moment is scaled on the host accordingly, so
// the transforms are additions only.
// (f_{-1}, f_0, f_{+1}) -> (sum f, sum e f, sum e^2 f) in place.
template <typename CT>
__device__ __forceinline__ void fwd3(CT& a, CT& b, CT& c) {
  const CT s = a + c, t = c - a;
  a = b + s; b = t; c = s;
}
// inverse of fwd3
template <typename CT>
__device__ __forceinline__ void inv3(CT& a, CT& b, CT& c) {
  const CT r = c, t = b, m0 = a;
  a = CT(0.5) * (r - t); c = CT(0.5) * (r + t); b = m0 - r;
}
// index moments about velocity u (in index units u / c): kappa_k = sum (e - u)^k f
template <typename CT>
__device__ __forceinline__ void shift3(CT& m0, CT& m1, CT& m2, CT u) {
  m2 = m2 - CT(2) * u * m1 + u * u * m0;
  m1 = m1 - u * m0;
}
template <typename CT>
__device__ __forceinline__ void unshift3(CT& k0, CT& k1, CT& k2, CT u) {
  k2 = k2 + CT(2) * u * k1 + u * u * k0;
  k1 = k1 + u * k0;
}

template <int LAT, typename CT> struct Cube {
  static constexpr int NZ = Lat<LAT>::NZ;
  CT v[3][3][NZ];

  __device__ __forceinline__ void forward() {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c) fwd3(v[0][b][c], v[1][b][c], v[2][b][c]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < NZ; ++c) fwd3(v[a][0][c], v[a][1][c], v[a][2][c]);
    if constexpr (NZ == 3) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) fwd3(v[a][b][0], v[a][b][1], v[a][b][2]);
    }
  }
  __device__ __forceinline__ void inverse() {
    if constexpr (NZ == 3) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) inv3(v[a][b][0], v[a][b][1], v[a][b][2]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < NZ; ++c) inv3(v[a][0][c], v[a][1][c], v[a][2][c]);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c) inv3(v[0][b][c], v[1][b][c], v[2][b][c]);
  }
  template <bool BACK>
  __device__ __forceinline__ void shift(const CT u[3]) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c)
        BACK ? unshift3(v[0][b][c], v[1][b][c], v[2][b][c], u[0]) : shift3(v[0][b][c], v[1][b][c], v[2][b][c], u[0]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < NZ; ++c)
        BACK ? unshift3(v[a][0][c], v[a][1][c], v[a][2][c], u[1]) : shift3(v[a][0][c], v[a][1][c], v[a][2][c], u[1]);
    if constexpr (NZ == 3) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          BACK ? unshift3(v[a][b][0], v[a][b][1], v[a][b][2], u[2]) : shift3(v[a][b][0], v[a][b][1], v[a][b][2], u[2]);
    }
  }
};

// True for the eight rD3Q27 monomials that vanish on rD3Q19.
template <int LAT>
__device__ __forceinline__ constexpr bool absent(int a, int b, int c) {
  return LAT == LAT_D3Q19 && a > 0 && b > 0 && c > 0;
}

// Index moment (a, b, c) of g^eq(A, B, M) (Eqs. 3-3/3-4), with B and M given
// in index units (Bh_a = B_a / c_a, Mh_ab = M_ab / (c_a c_b)).  With the
// 1-D weight moments mu(0) = 1, mu(1) = 0, mu_a(2) = c_s^2 / c_a^2:
//   mh = A prod mu + sum_al [a_al = 1] Bh_al prod_{be != al} mu
//      + sum_al [a_al = 2] Mh_alal prod_{be != al} mu
//      + sum_{al < be} [a_al = a_be = 1] Mh_albe prod_{ga} mu.
// Exact for the tensor-product weights of rD2Q9 and of rD3Q27 with the
// omega_19 chosen on the host; rD3Q19 (omega_19 = 0) adds
// -c_s^4 M_gg / (c_g^2 - c_s^2) to the physical (2,2,0)-type moments (g
// the axis with exponent 0), q19h[g] carrying the index scaling.
// Mh is packed xx, yy, zz, xy, xz, yz.
template <int LAT, typename CT>
__device__ __forceinline__ CT meq_moment(int a, int b, int c, CT A, const CT B[3], const CT M[6],
                                         const KParams<CT>& p) {
  auto mx = [&](int k) -> CT { return k == 0 ? CT(1) : (k == 1 ? CT(0) : p.mu2[0]); };
  auto my = [&](int k) -> CT { return k == 0 ? CT(1) : (k == 1 ? CT(0) : p.mu2[1]); };
  auto mz = [&](int k) -> CT { return k == 0 ? CT(1) : (k == 1 ? CT(0) : p.mu2[2]); };
  CT r = CT(0);
  if (a != 1 && b != 1 && c != 1) r = A * mx(a) * my(b) * mz(c);
  if (a == 1 && b != 1 && c != 1) r += B[0] * my(b) * mz(c);
  if (b == 1 && a != 1 && c != 1) r += B[1] * mx(a) * mz(c);
  if (c == 1 && a != 1 && b != 1) r += B[2] * mx(a) * my(b);
  if (a == 2 && b != 1 && c != 1) r += M[0] * my(b) * mz(c);
  if (b == 2 && a != 1 && c != 1) r += M[1] * mx(a) * mz(c);
  if (c == 2 && a != 1 && b != 1) r += M[2] * mx(a) * my(b);
  if (a == 1 && b == 1 && c != 1) r += M[3] * mz(c);
  if (a == 1 && c == 1 && b != 1) r += M[4] * my(b);
  if (b == 1 && c == 1 && a != 1) r += M[5] * mx(a);
  if (LAT == LAT_D3Q19) {
    if (a == 2 && b == 2 && c == 0) r -= p.q19h[2] * M[2];
    if (a == 2 && b == 0 && c == 2) r -= p.q19h[1] * M[1];
    if (a == 0 && b == 2 && c == 2) r -= p.q19h[0] * M[0];
  }
  return r;
}

// S x for the entry (a, b, c) (Eq. 5-1 block structure in index units): the
// order-2 diagonal entries use the dense block, scaled to index units on the
// host (s2h = D^-1 S_2 D).
template <int LAT, typename CT>
__device__ __forceinline__ CT relax(int a, int b, int c, const CT (&X)[3][3][Lat<LAT>::NZ],
                                    const KParams<CT>& p) {
  const int o = a + b + c;
  if (absent<LAT>(a, b, c)) return CT(0);
  if (o == 0) return p.s0 * X[0][0][0];
  if (o == 1) return p.s1[a == 1 ? 0 : (b == 1 ? 1 : 2)] * X[a][b][c];
  if (o == 2 && (a == 2 || b == 2 || c == 2)) {
    const int r = a == 2 ? 0 : (b == 2 ? 1 : 2);
    CT s = p.s2h[r][0] * X[2][0][0] + p.s2h[r][1] * X[0][2][0];
    if constexpr (Lat<LAT>::NZ == 3) s += p.s2h[r][2] * X[0][0][2];
    return s;
  }
  if (o == 2) return p.soff[(a == 1 && b == 1) ? 0 : ((a == 1) ? 1 : 2)] * X[a][b][c];
  return p.sfree * X[a][b][c];
}

// Equilibrium arguments in index units and the velocity (u / c) about
// which central moments are taken.
template <typename CT>
struct Macro {
  CT dA;      // A - rho0 (density or phi deviation)
  CT B[3];    // B_a / c_a
  CT M[6];    // M_ab / (c_a c_b): xx yy zz xy xz yz
  CT u[3];    // u_a / c_a: fluid (NSE) or advection (NCDE) velocity
  CT rho;     // density or phi
};

// A, B, M of the model for density (or phi) rho and index velocity uh.
template <typename CT>
__device__ __forceinline__ void eq_args(Macro<CT>& r, CT rho, const CT uh[3], const KParams<CT>& p) {
  CT fb, fc;
  if (p.kind == KIND_NSE) { fb = rho; fc = rho; }                    // g^eq(rho, rho u, rho u u)
  else if (p.kind == KIND_NSE_HELUO) { fb = p.rho0; fc = p.rho0; }   // g^eq(rho, rho0 u, rho0 u u)
  else if (p.kind == KIND_NCDE_LINEAR) { fb = rho; fc = rho; }       // B = u phi, C = u u phi
  else { fb = CT(0.5) * rho * rho; fc = rho * rho * rho * CT(1.0 / 3.0); }  // B = u phi^2/2, C = u u phi^3/3
#pragma unroll
  for (int al = 0; al < 3; ++al) { r.u[al] = uh[al]; r.B[al] = fb * uh[al]; }
  r.M[0] = fc * uh[0] * uh[0]; r.M[1] = fc * uh[1] * uh[1]; r.M[2] = fc * uh[2] * uh[2];
  r.M[3] = fc * uh[0] * uh[1]; r.M[4] = fc * uh[0] * uh[2]; r.M[5] = fc * uh[1] * uh[2];
}

// Conserved fields from the index moments (Eqs. 2-4-1 / 2-4-2).
template <int D, typename CT>
__device__ __forceinline__ Macro<CT> macroscopic(CT m000, const CT jh[3], const KParams<CT>& p) {
  Macro<CT> r;
  const CT hdt = CT(0.5) * p.dt;
  const CT drho = m000 + hdt * p.source;
  r.dA = drho;
  r.rho = p.rho0 + drho;
  CT uh[3];
  if (p.kind == KIND_NSE || p.kind == KIND_NSE_HELUO) {
    const CT inv = CT(1) / (p.kind == KIND_NSE ? r.rho : p.rho0);
#pragma unroll
    for (int al = 0; al < 3; ++al) uh[al] = (al < D) ? (jh[al] + hdt * p.fh[al]) * inv : CT(0);
  } else {
#pragma unroll
    for (int al = 0; al < 3; ++al) uh[al] = p.advh[al];
  }
  eq_args(r, r.rho, uh, p);
  return r;
}

// Collision of one node in moment space, Eq. (2-2-3):
//   m* - m0 = m(delta) + dt (m_G + m_F) - S (m^ne + dt m_F / 2),
// central variant: S replaced by N(u)^-1 Sbar N(u) (Eq. 5-1-2).
template <int LAT, typename CT, bool CENTRAL, bool FORCED>
__device__ __forceinline__ void collide(Cube<LAT, CT>& q, const KParams<CT>& p) {
  constexpr int D = Lat<LAT>::D, NZ = Lat<LAT>::NZ;
  q.forward();
  CT jh[3] = {q.v[1][0][0], q.v[0][1][0], CT(0)};
  if constexpr (NZ == 3) jh[2] = q.v[0][0][NZ - 2];
  const Macro<CT> mc = macroscopic<D>(q.v[0][0][0], jh, p);

  // forcing moments (index units): F = g^eq(Sbar, Fbar, -c_s^2 Sbar I) (NSE)
  // or omega S (NCDE); G = g^eq(0, 0, M_2G), M_2G = (I - S_2/2)(u F + F u +
  // c_s^2 Sbar I) (NSE), or G = g^eq(0, (I - S_1/2) B' S, 0) (NCDE).
  CT FA = CT(0), FB[3] = {CT(0), CT(0), CT(0)}, FM[6] = {CT(0), CT(0), CT(0), CT(0), CT(0), CT(0)};
  CT GB[3] = {CT(0), CT(0), CT(0)}, GM[6] = {CT(0), CT(0), CT(0), CT(0), CT(0), CT(0)};
  const bool nse = p.kind == KIND_NSE || p.kind == KIND_NSE_HELUO;
  if constexpr (FORCED) {
    FA = p.source;
    if (nse) {
#pragma unroll
      for (int al = 0; al < 3; ++al) { FB[al] = p.fh[al]; FM[al] = -p.source * p.mu2[al]; }
      CT Y[6];
#pragma unroll
      for (int al = 0; al < 3; ++al) Y[al] = CT(2) * mc.u[al] * p.fh[al] + p.source * p.mu2[al];
      Y[3] = mc.u[0] * p.fh[1] + p.fh[0] * mc.u[1];
      Y[4] = mc.u[0] * p.fh[2] + p.fh[0] * mc.u[2];
      Y[5] = mc.u[1] * p.fh[2] + p.fh[1] * mc.u[2];
#pragma unroll
      for (int r = 0; r < D; ++r) {
        CT s = CT(0);
#pragma unroll
        for (int k = 0; k < D; ++k) s += p.s2h[r][k] * Y[k];
        GM[r] = Y[r] - CT(0.5) * s;
      }
      GM[3] = (CT(1) - CT(0.5) * p.soff[0]) * Y[3];
      GM[4] = (CT(1) - CT(0.5) * p.soff[1]) * Y[4];
      GM[5] = (CT(1) - CT(0.5) * p.soff[2]) * Y[5];
    } else {
      const CT bp = p.kind == KIND_NCDE_LINEAR ? CT(1) : mc.rho;   // B' = u bp
#pragma unroll
      for (int al = 0; al < 3; ++al) GB[al] = (CT(1) - CT(0.5) * p.s1[al]) * p.advh[al] * bp * p.source;
    }
  }
  const CT zero3[3] = {CT(0), CT(0), CT(0)};
  const CT zero6[6] = {CT(0), CT(0), CT(0), CT(0), CT(0), CT(0)};
  const CT hdt = CT(0.5) * p.dt;

  // X = m^ne + dt m_F / 2 ; q becomes m(delta) + dt (m_G + m_F)
  CT X[3][3][NZ];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c) {
        if (absent<LAT>(a, b, c)) { X[a][b][c] = CT(0); continue; }
        const CT meq = meq_moment<LAT>(a, b, c, mc.dA, mc.B, mc.M, p);
        X[a][b][c] = q.v[a][b][c] - meq;
        if constexpr (FORCED) {
          const CT mF = meq_moment<LAT>(a, b, c, FA, FB, FM, p);
          const CT mG = nse ? meq_moment<LAT>(a, b, c, CT(0), zero3, GM, p)
                            : meq_moment<LAT>(a, b, c, CT(0), GB, zero6, p);
          X[a][b][c] += hdt * mF;
          q.v[a][b][c] += p.dt * (mG + mF);
        }
      }
  if constexpr (CENTRAL) {
    Cube<LAT, CT> k;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) k.v[a][b][c] = X[a][b][c];
    k.template shift<false>(mc.u);
    CT SX[3][3][NZ];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) SX[a][b][c] = relax<LAT>(a, b, c, k.v, p);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) k.v[a][b][c] = SX[a][b][c];
    k.template shift<true>(mc.u);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) q.v[a][b][c] -= k.v[a][b][c];
  } else {
    CT SX[3][3][NZ];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) SX[a][b][c] = relax<LAT>(a, b, c, X, p);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) q.v[a][b][c] -= SX[a][b][c];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c)
        if (absent<LAT>(a, b, c)) q.v[a][b][c] = CT(0);
  q.inverse();
}

template <int LAT>
__device__ __forceinline__ constexpr int zi(int ez) { return Lat<LAT>::NZ == 3 ? ez + 1 : 0; }

// ------------------------------------------------------------------ kernels
// One time step: pull gather from fin (post-collision of the previous step,
// x - e_j), collide, store the post-collision state of node x in fout.
template <int LAT, typename ST, typename CT, bool CENTRAL, bool FORCED>
__global__ void __launch_bounds__(128) step_kernel(const ST* __restrict__ fin, ST* __restrict__ fout,
                                                   const KParams<CT> p) {
  using L = Lat<LAT>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.nx) return;
  const Nbr nb(x, y, z, p.nx, p.ny, p.nz);
  const size_t N = p.N;
  Cube<LAT, CT> q;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < L::NZ; ++c) q.v[a][b][c] = CT(0);
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    const int sx = Nbr::up(ex, nb.xm, nb.x0, nb.xp);
    const int sy = Nbr::up(ey, nb.ym, nb.y0, nb.yp);
    const int sz = Nbr::up(ez, nb.zm, nb.z0, nb.zp);
    const size_t idx = (size_t(sz) * p.ny + sy) * p.nx + sx;
    q.v[ex + 1][ey + 1][zi<LAT>(ez)] = load_st<ST, CT>(fin + j * N + idx) * p.sinv[j];
  });
  collide<LAT, CT, CENTRAL, FORCED>(q, p);
  const size_t own = (size_t(z) * p.ny + y) * p.nx + x;
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    store_st<ST, CT>(fout + j * N + own, q.v[ex + 1][ey + 1][zi<LAT>(ez)] * p.sc[j]);
  });
}

// ------------------------------------------------------------------ paired storage access
template <typename ST> struct Pair;
template <> struct Pair<double> { using T = double2; };
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<__half> { using T = __half2; };
template <> struct Pair<__nv_bfloat16> { using T = __nv_bfloat162; };

template <typename ST, typename CT>
__device__ __forceinline__ void load_pair(const ST* p, CT& lo, CT& hi) {
  const auto v = __ldg(reinterpret_cast<const typename Pair<ST>::T*>(p));
  lo = static_cast<CT>(v.x); hi = static_cast<CT>(v.y);
}
template <>
__device__ __forceinline__ void load_pair<__half, float>(const __half* p, float& lo, float& hi) {
  const float2 v = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
  lo = v.x; hi = v.y;
}
template <>
__device__ __forceinline__ void load_pair<__nv_bfloat16, float>(const __nv_bfloat16* p, float& lo, float& hi) {
  const float2 v = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
  lo = v.x; hi = v.y;
}
template <typename ST, typename CT>
__device__ __forceinline__ void store_pair(ST* p, CT lo, CT hi) {
  typename Pair<ST>::T v;
  v.x = static_cast<ST>(lo); v.y = static_cast<ST>(hi);
  *reinterpret_cast<typename Pair<ST>::T*>(p) = v;
}
template <>
__device__ __forceinline__ void store_pair<__half, float>(__half* p, float lo, float hi) {
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(lo, hi);
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16, float>(__nv_bfloat16* p, float lo, float hi) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(lo, hi);
}

// One time step, two x-adjacent nodes (x0, x0 + 1) per thread, x0 even;
// requires nx even so that every pair is aligned to twice the element size.
// A direction with e_x = 0 is one aligned pair load.  For e_x = +1 the
// thread needs (x0 - 1, x0): x0 is the low half of its own aligned pair and
// x0 - 1 the high half of the lane below (warp shuffle); lane 0 loads it.
// For e_x = -1 it needs (x0 + 1, x0 + 2) symmetrically from the lane above,
// the last lane of a warp or of a row loading x0 + 2 itself (periodic wrap).
// Every lane takes part in the shuffles; lanes past the row end clamp their
// loads to the last pair and store nothing.
template <int LAT, typename ST, typename CT, bool CENTRAL, bool FORCED>
__global__ void __launch_bounds__(128) step_kernel_x2(const ST* __restrict__ fin, ST* __restrict__ fout,
                                                      const KParams<CT> p) {
  using L = Lat<LAT>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int x0 = 2 * t;
  const bool active = x0 < p.nx;
  const int xc = active ? x0 : p.nx - 2;
  const int lane = threadIdx.x & 31;
  const int y = blockIdx.y, z = blockIdx.z;
  const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
  const bool fix_lo = lane == 0;                       // needs x0 - 1 from memory
  const bool fix_hi = lane == 31 || xc + 2 >= p.nx;    // needs x0 + 2 from memory
  const int x_lo = xc == 0 ? p.nx - 1 : xc - 1;
  const int x_hi = xc + 2 >= p.nx ? 0 : xc + 2;
  const size_t N = p.N;
  Cube<LAT, CT> qa, qb;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < L::NZ; ++c) { qa.v[a][b][c] = CT(0); qb.v[a][b][c] = CT(0); }
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    const int sy = Nbr::up(ey, ym, y, yp);
    const int sz = Nbr::up(ez, zm, z, zp);
    const ST* row = fin + j * N + (size_t(sz) * p.ny + sy) * p.nx;
    CT lo, hi, va, vb;
    load_pair<ST, CT>(row + xc, lo, hi);
    if constexpr (ex == 0) {
      va = lo; vb = hi;
    } else if constexpr (ex == 1) {
      CT prev = __shfl_up_sync(0xffffffffu, hi, 1);
      if (fix_lo) prev = load_st<ST, CT>(row + x_lo);
      va = prev; vb = lo;
    } else {
      CT next = __shfl_down_sync(0xffffffffu, lo, 1);
      if (fix_hi) next = load_st<ST, CT>(row + x_hi);
      va = hi; vb = next;
    }
    qa.v[ex + 1][ey + 1][zi<LAT>(ez)] = va * p.sinv[j];
    qb.v[ex + 1][ey + 1][zi<LAT>(ez)] = vb * p.sinv[j];
  });
  collide<LAT, CT, CENTRAL, FORCED>(qa, p);
  collide<LAT, CT, CENTRAL, FORCED>(qb, p);
  if (!active) return;
  const size_t own = (size_t(z) * p.ny + y) * p.nx + x0;
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    store_pair<ST, CT>(fout + j * N + own, qa.v[ex + 1][ey + 1][zi<LAT>(ez)] * p.sc[j],
                       qb.v[ex + 1][ey + 1][zi<LAT>(ez)] * p.sc[j]);
  });
}

}  // namespace rmrt
