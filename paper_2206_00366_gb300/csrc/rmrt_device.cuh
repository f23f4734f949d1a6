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
// sc_j the power of two nearest 1/omega_j for FP16 and E3M12 storage (exact
// to apply and to undo; for E3M12 also times 2^(bias - 127), see E3M12
// below) and 1 for the others;
// every moment below is a moment of delta_j = fbar_j - omega_j rho0, so the
// rest state never enters the arithmetic (m(omega rho0) = m^eq(rho0, 0, 0)).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>
#include <utility>

#include "rmrt_params.h"
#include "rmrt_tuning.h"

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
// rD2Q5 and rD3Q7 (Remark I of Sec. III): the rest and axis directions,
// the first 5 of rD2Q9 and the first 7 of rD3Q27.
template <> struct Lat<LAT_D2Q5> {
  static constexpr int D = 2, Q = 5, NZ = 1;
  static constexpr int EX[5] = {0, 1, 0, -1, 0};
  static constexpr int EY[5] = {0, 0, 1, 0, -1};
  static constexpr int EZ[5] = {0, 0, 0, 0, 0};
};
template <> struct Lat<LAT_D3Q7> : Dirs27 {
  static constexpr int D = 3, Q = 7, NZ = 3;
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
// E3M12: a 16-bit float with a sign bit, 3 exponent bits (bias 5) and 12
// mantissa bits, with subnormals: 4x the resolution of FP16 for magnitudes
// of the scaled deviation in [2^-4, 8), FP16's absolute resolution 2^-16
// below, and saturation at 8 - 2^-10 (counted by the check kernel).  A
// value x is held in FP32 as w = x * 2^(5 - 127) (the factor is folded into
// the storage scale sc_j, its inverse into sinv_j), which places the E3M12
// code of x, normal or subnormal, in bits 11..25 of w: decoding is a shift,
// encoding a rounding at bit 11 and a shift.  The FP32 arithmetic that meets
// w is compiled without flush-to-zero, so subnormal w are exact.
struct E3M12 {
  unsigned short b;
};
constexpr int E3M12_BIAS = 5;
constexpr unsigned E3M12_MAX_W = 0x03FFF800u;    // FP32 bits of the largest code's w

__device__ __forceinline__ float e3m12_decode(unsigned code) {
  return __uint_as_float(((code & 0x7FFFu) << 11) | ((code & 0x8000u) << 16));
}
// Two codes of one 32-bit word (low half first) to FP32.
__device__ __forceinline__ float2 e3m12_decode2(unsigned w) {
  return make_float2(__uint_as_float(((w & 0x7FFFu) << 11) | ((w & 0x8000u) << 16)),
                     __uint_as_float(((w >> 5) & 0x03FFF800u) | (w & 0x80000000u)));
}
// |w| bits plus the rounding increment, saturated at the largest code, as a
// code magnitude in bits 11..25.
__device__ __forceinline__ unsigned e3m12_mag(unsigned u, unsigned add) {
  return min((u & 0x7FFFFFFFu) + add, 0x03FFFFFFu);
}
// Round to nearest, ties to even.
__device__ __forceinline__ unsigned e3m12_encode_rn(float w) {
  const unsigned u = __float_as_uint(w);
  const unsigned a = e3m12_mag(u, 0x3FFu + ((u >> 11) & 1u));
  return (a >> 11) | ((u >> 16) & 0x8000u);
}
// Stochastic rounding of two values into one word (x low half, y high
// half): r supplies 11 random bits per value (bits 0..10 and 16..26); adding
// them below bit 11 and truncating rounds up with probability equal to the
// discarded fraction of a unit in the last place.
__device__ __forceinline__ unsigned e3m12_encode2_sr(float x, float y, unsigned r) {
  const unsigned ux = __float_as_uint(x), uy = __float_as_uint(y);
  const unsigned ax = e3m12_mag(ux, r & 0x7FFu), ay = e3m12_mag(uy, (r >> 16) & 0x7FFu);
  return (ax >> 11) | ((ux >> 16) & 0x8000u) | ((ay << 5) & 0x7FFF0000u) | (uy & 0x80000000u);
}

// Random bits for stochastic rounding: one 32-bit hash of the step's seed
// and the thread's first node, and from it word K = hash * (an odd constant
// per K), one integer multiply per word.  Multiplying by an odd number is a
// bijection, so every word is uniformly distributed over the nodes and
// steps, and the words of one thread differ by their multipliers.  The
// rounding only needs bits that are uniform and unrelated to the values
// rounded; the sequence is reproducible for a given step and grid.
struct SrBits {
  unsigned s;
  __device__ __forceinline__ explicit SrBits(unsigned seed, unsigned node) {
    unsigned x = seed ^ (node * 0x9E3779B1u);
    x ^= x >> 16; x *= 0x7FEB352Du; x ^= x >> 15; x *= 0x846CA68Bu; x ^= x >> 16;
    s = x;
  }
  template <int K>
  __device__ __forceinline__ unsigned word() const {
    return s * (0x9E3779B1u + 2u * unsigned(K) * 0x632BE5ABu);
  }
};

template <typename ST, typename CT> __device__ __forceinline__ CT load_st(const ST* p) {
  return static_cast<CT>(__ldg(p));
}
template <> __device__ __forceinline__ float load_st<__half, float>(const __half* p) {
  return __half2float(__ldg(p));
}
template <> __device__ __forceinline__ float load_st<__nv_bfloat16, float>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float load_st<E3M12, float>(const E3M12* p) {
  return e3m12_decode(__ldg(reinterpret_cast<const unsigned short*>(p)));
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
template <> __device__ __forceinline__ void store_st<E3M12, float>(E3M12* p, float v) {
  p->b = (unsigned short)e3m12_encode_rn(v);
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

// ------------------------------------------------------------------ value types
// The collision is written once for a value type V with scalar parameter
// type S = Scalar<V>: V = float or double (one node per value), or F2 (two
// nodes per value, FP32).  F2 arithmetic maps onto the packed FP32
// instructions of sm_100-class GPUs (__fadd2_rn, __fmul2_rn, __ffma2_rn),
// so a thread that owns two nodes spends one instruction per operation.
struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ F2(float2 x) : v(x) {}
  __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ F2(double s) : v(make_float2(float(s), float(s))) {}
  __device__ __forceinline__ F2(int s) : v(make_float2(float(s), float(s))) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { a = a + b; return a; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { a = a - b; return a; }

template <typename V> struct ScalarOf { using T = V; };
template <> struct ScalarOf<F2> { using T = float; };
template <typename V> using Scalar = typename ScalarOf<V>::T;

__device__ __forceinline__ float fmav(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmav(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ F2 fmav(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

// 1 / x: CUDA's fast single-precision reciprocal for FP32 (its error is far
// below the FP32 storage rounding), exact division for FP64.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ F2 recip(F2 x) { return F2(__frcp_rn(x.v.x), __frcp_rn(x.v.y)); }

// ------------------------------------------------------------------ 1-D transforms
// The moments are index moments mh_abc = sum_j e_jx^a e_jy^b e_jz^c f_j; the
// physical raw moments of Eq. (5-2) are m_abc = c_x^a c_y^b c_z^c mh_abc.
// Every constant that meets a moment is scaled on the host accordingly, so
// the transforms are additions only.
// (f_{-1}, f_0, f_{+1}) -> (sum f, sum e f, sum e^2 f) in place.
template <typename V>
__device__ __forceinline__ void fwd3(V& a, V& b, V& c) {
  const V s = a + c, t = c - a;
  a = b + s; b = t; c = s;
}
// inverse of fwd3
template <typename V>
__device__ __forceinline__ void inv3(V& a, V& b, V& c) {
  const V r = c, t = b, m0 = a;
  a = (r - t) * V(0.5f); c = (r + t) * V(0.5f); b = m0 - r;
}
// index moments about velocity u (in index units u / c): kappa_k = sum (e - u)^k f
template <typename V>
__device__ __forceinline__ void shift3(V& m0, V& m1, V& m2, V u) {
  m2 = fmav(u * u, m0, fmav(V(-2.0f) * u, m1, m2));
  m1 = fmav(-u, m0, m1);
}
template <typename V>
__device__ __forceinline__ void unshift3(V& k0, V& k1, V& k2, V u) {
  k2 = fmav(u * u, k0, fmav(V(2.0f) * u, k1, k2));
  k1 = fmav(u, k0, k1);
}

template <int LAT, typename V> struct Cube {
  static constexpr int NZ = Lat<LAT>::NZ;
  V v[3][3][NZ];

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
  __device__ __forceinline__ void shift(const V u[3]) {
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

// True for the cube moments the lattice does not carry: the eight rD3Q27
// monomials that vanish on rD3Q19, and on rD2Q5/rD3Q7 every monomial with
// two or more nonzero exponents.
template <int LAT>
__device__ __forceinline__ constexpr bool absent(int a, int b, int c) {
  if (LAT == LAT_D2Q5 || LAT == LAT_D3Q7) return (a > 0) + (b > 0) + (c > 0) >= 2;   // axis-only lattices
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
// Scalar type of a parameter block (KParams<S> or any struct with the same
// field names).
template <typename P>
using PScalar = typename std::remove_cv<typename std::remove_reference<decltype(P::rho0)>::type>::type;

// Hermite moments from raw moments along every axis (BACK: the inverse):
// with P_2(e) = e^2 - mu (mu = c_s^2 / c_a^2 in index units), the 1-D map
// (m0, m1, m2) -> (m0, m1, m2 - mu m0) is unit lower-triangular.
template <bool BACK, int LAT, typename V, typename P>
__device__ __forceinline__ void hermite_axes(Cube<LAT, V>& q, const P& p) {
  using S = PScalar<P>;
  constexpr int NZ = Lat<LAT>::NZ;
  const S sg = BACK ? S(1) : S(-1);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < NZ; ++c) q.v[2][b][c] = fmav(q.v[0][b][c], V(sg * p.mu2[0]), q.v[2][b][c]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < NZ; ++c) q.v[a][2][c] = fmav(q.v[a][0][c], V(sg * p.mu2[1]), q.v[a][2][c]);
  if constexpr (NZ == 3) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) q.v[a][b][2] = fmav(q.v[a][b][0], V(sg * p.mu2[2]), q.v[a][b][2]);
  }
}

template <int LAT, typename V, typename P>
__device__ __forceinline__ V meq_moment(int a, int b, int c, V A, const V B[3], const V M[6], const P& p) {
  using S = PScalar<P>;
  auto mx = [&](int k) -> S { return k == 0 ? S(1) : (k == 1 ? S(0) : p.mu2[0]); };
  auto my = [&](int k) -> S { return k == 0 ? S(1) : (k == 1 ? S(0) : p.mu2[1]); };
  auto mz = [&](int k) -> S { return k == 0 ? S(1) : (k == 1 ? S(0) : p.mu2[2]); };
  // term * factor with the factor folded away when it is exactly 1
  auto acc = [&](V r, V term, int f0, int f1, S fac) -> V {
    return (f0 == 0 && f1 == 0) ? r + term : fmav(term, V(fac), r);
  };
  V r = V(0.0f);
  if (a != 1 && b != 1 && c != 1) {
    const int n2 = (a == 2) + (b == 2) + (c == 2);
    r = n2 == 0 ? A : A * V(mx(a) * my(b) * mz(c));
  }
  if (a == 1 && b != 1 && c != 1) r = acc(r, B[0], b, c, my(b) * mz(c));
  if (b == 1 && a != 1 && c != 1) r = acc(r, B[1], a, c, mx(a) * mz(c));
  if (c == 1 && a != 1 && b != 1) r = acc(r, B[2], a, b, mx(a) * my(b));
  if (a == 2 && b != 1 && c != 1) r = acc(r, M[0], b, c, my(b) * mz(c));
  if (b == 2 && a != 1 && c != 1) r = acc(r, M[1], a, c, mx(a) * mz(c));
  if (c == 2 && a != 1 && b != 1) r = acc(r, M[2], a, b, mx(a) * my(b));
  if (a == 1 && b == 1 && c != 1) r = acc(r, M[3], c, 0, mz(c));
  if (a == 1 && c == 1 && b != 1) r = acc(r, M[4], b, 0, my(b));
  if (b == 1 && c == 1 && a != 1) r = acc(r, M[5], a, 0, mx(a));
  if (LAT == LAT_D3Q19) {
    if (a == 2 && b == 2 && c == 0) r = fmav(M[2], V(-p.q19h[2]), r);
    if (a == 2 && b == 0 && c == 2) r = fmav(M[1], V(-p.q19h[1]), r);
    if (a == 0 && b == 2 && c == 2) r = fmav(M[0], V(-p.q19h[0]), r);
  }
  return r;
}

// Rate of a diagonal moment class (Eq. 5-1 block structure in index units);
// the order-2 diagonal entries instead use the dense block s2h = D^-1 S_2 D.
template <typename P>
__device__ __forceinline__ PScalar<P> diag_rate(int a, int b, int c, const P& p) {
  const int o = a + b + c;
  if (o == 0) return p.s0;
  if (o == 1) return p.s1[a == 1 ? 0 : (b == 1 ? 1 : 2)];
  if (o == 2) return p.soff[(a == 1 && b == 1) ? 0 : ((a == 1) ? 1 : 2)];
  return p.sfree;
}
template <int a, int b, int c>
__device__ __forceinline__ constexpr bool dense_block() {
  return a + b + c == 2 && (a == 2 || b == 2 || c == 2);
}

// out = out - S X (ACC) or out = S X (!ACC).  For the NSE family orders 0
// and 1 are conserved: X vanishes there (Eq. 4-18-1 with the dt F / 2 terms
// of Eq. 2-4-2), so s_0 and S_1 act on zero and are skipped.
template <int LAT, bool NSE, bool ACC, typename V, typename P>
__device__ __forceinline__ void relax(V (&out)[3][3][Lat<LAT>::NZ], const V (&X)[3][3][Lat<LAT>::NZ],
                                      const P& p) {
  using S = PScalar<P>;
  constexpr int NZ = Lat<LAT>::NZ;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c) {
        const int o = a + b + c;
        if (absent<LAT>(a, b, c) || (NSE && o < 2)) {
          if (!ACC) out[a][b][c] = V(0.0f);
          continue;
        }
        if (o == 2 && (a == 2 || b == 2 || c == 2)) {
          const int r = a == 2 ? 0 : (b == 2 ? 1 : 2);
          V t = ACC ? out[a][b][c] : V(0.0f);
          const S sg = ACC ? S(-1) : S(1);
          t = fmav(X[2][0][0], V(sg * p.s2h[r][0]), t);
          t = fmav(X[0][2][0], V(sg * p.s2h[r][1]), t);
          if constexpr (NZ == 3) t = fmav(X[0][0][2], V(sg * p.s2h[r][2]), t);
          out[a][b][c] = t;
        } else {
          const S s = diag_rate<P>(a, b, c, p);
          out[a][b][c] = ACC ? fmav(X[a][b][c], V(-s), out[a][b][c]) : X[a][b][c] * V(s);
        }
      }
}

// Equilibrium arguments in index units and the velocity (u / c) about
// which central moments are taken.
template <typename V>
struct Macro {
  V dA;      // A - rho0 (density or phi deviation)
  V B[3];    // B_a / c_a
  V M[6];    // M_ab / (c_a c_b): xx yy zz xy xz yz
  V u[3];    // u_a / c_a: fluid (NSE) or advection (NCDE) velocity
  V rho;     // density or phi
};

// A, B, M of the model for density (or phi) rho and index velocity uh.
template <typename CT>
__device__ __forceinline__ void eq_args(Macro<CT>& r, CT rho, const CT uh[3], const KParams<CT>& p) {
  CT fb, fc;
  if (p.kind == KIND_NSE) { fb = rho; fc = rho; }                    // g^eq(rho, rho u, rho u u)
  else if (p.kind == KIND_NSE_HELUO) { fb = p.rho0; fc = p.rho0; }   // g^eq(rho, rho0 u, rho0 u u)
  else if (p.kind == KIND_NCDE_LINEAR) { fb = rho; fc = rho; }       // B = u phi, C = u u phi
  else if (p.kind == KIND_NCDE_QUAD) { fb = CT(0.5) * rho * rho; fc = rho * rho * rho * CT(1.0 / 3.0); }  // B = u phi^2/2, C = u u phi^3/3
  else { fb = p.kind == KIND_NCDE_SIMPLE_LINEAR ? rho : CT(0.5) * rho * rho; fc = CT(0); }   // Eq. (4-16): C = 0
#pragma unroll
  for (int al = 0; al < 3; ++al) { r.u[al] = uh[al]; r.B[al] = fb * uh[al]; }
  r.M[0] = fc * uh[0] * uh[0]; r.M[1] = fc * uh[1] * uh[1]; r.M[2] = fc * uh[2] * uh[2];
  r.M[3] = fc * uh[0] * uh[1]; r.M[4] = fc * uh[0] * uh[2]; r.M[5] = fc * uh[1] * uh[2];
}

// Conserved fields from the index moments (Eqs. 2-4-1 / 2-4-2).  NSE: the
// family of the NSE and He-Luo equilibria; otherwise the two NCDE kinds.
template <int D, bool NSE, typename V, typename P>
__device__ __forceinline__ Macro<V> macroscopic(V m000, const V jh[3], const P& p) {
  using S = PScalar<P>;
  Macro<V> r;
  const S hdt = S(0.5) * p.dt;
  const V drho = m000 + V(hdt * p.source);
  r.dA = drho;
  r.rho = V(p.rho0) + drho;
  V uh[3], fb, fc;
  if constexpr (NSE) {
    const bool heluo = p.kind == KIND_NSE_HELUO;
    const V inv = heluo ? V(S(1) / p.rho0) : recip(r.rho);
#pragma unroll
    for (int al = 0; al < 3; ++al) uh[al] = (al < D) ? fmav(V(hdt * p.fh[al]), inv, jh[al] * inv) : V(0.0f);
    fb = heluo ? V(p.rho0) : r.rho;                    // g^eq(rho, rho u, rho u u) or (rho, rho0 u, rho0 u u)
    fc = fb;
  } else {
#pragma unroll
    for (int al = 0; al < 3; ++al) uh[al] = V(p.advh[al]);
    const bool lin = p.kind == KIND_NCDE_LINEAR || p.kind == KIND_NCDE_SIMPLE_LINEAR;   // B = u phi
    fb = lin ? r.rho : V(0.5f) * r.rho * r.rho;        // B = u phi^2/2
    if (p.kind >= KIND_NCDE_SIMPLE_LINEAR) fc = V(0.0f);   // Eq. (4-16): C = 0 (linear EDF)
    else fc = lin ? r.rho : r.rho * r.rho * r.rho * V(S(1.0 / 3.0));   // C = u u phi, u u phi^3/3
  }
#pragma unroll
  for (int al = 0; al < 3; ++al) { r.u[al] = uh[al]; r.B[al] = fb * uh[al]; }
  const V fu0 = fc * uh[0], fu1 = fc * uh[1];
  r.M[0] = fu0 * uh[0]; r.M[1] = fu1 * uh[1]; r.M[2] = fc * uh[2] * uh[2];
  r.M[3] = fu0 * uh[1]; r.M[4] = fu0 * uh[2]; r.M[5] = fu1 * uh[2];
  return r;
}

// The other bases for the NSE kinds, without a second cube of moments.
// With Mbar = T M (T unit lower-triangular by order: the central shift N(u)
// and/or the Hermite map, Eq. 5-1-1) and Sbar = s_free I + D, D nonzero only
// up to second order, the collision operator of Eq. (5-1-2) applied to the
// non-equilibrium moments X is s_free X + T^-1 D T X.  For the NSE family
// X vanishes at orders 0 and 1, so (T X) at second order is X's own second
// order (the shift and the Hermite map only add lower orders to it) and
// E = D T X = (Sbar_2 - s_free I) X_2 has second-order entries only.  T^-1
// is a tensor product of one 3 x 3 lower-triangular matrix per axis,
// G = [[1, 0, 0], [g1, 1, 0], [g2, g21, 1]]: central g1 = u, g2 = u^2,
// g21 = 2u; Hermite g1 = 0, g2 = mu, g21 = 0; central-Hermite g1 = u,
// g2 = u^2 + mu, g21 = 2u (index units, mu = c_s^2 / c_a^2).  So the step
// is the raw step at the single rate s_free minus T^-1 E, whose entries are
// sums of at most six products; moments the lattice does not carry are
// zeroed afterwards as in every basis.
template <int LAT, int BASIS, typename V, typename P>
__device__ __forceinline__ void subtract_transported(Cube<LAT, V>& q, const V (&X)[3][3][Lat<LAT>::NZ],
                                                     const V u[3], const P& p) {
  using S = PScalar<P>;
  constexpr int NZ = Lat<LAT>::NZ;
  constexpr bool SH = (BASIS & 1) != 0, HE = (BASIS & 2) != 0;
  // E = (Sbar_2 - s_free) X_2: the dense block on the normal moments, the
  // off-diagonal rates on the mixed ones
  const V x0 = X[2][0][0], x1 = X[0][2][0];
  const V x2 = NZ == 3 ? X[0][0][NZ - 1] : V(0.0f);
  V En[3];
#pragma unroll
  for (int r = 0; r < (NZ == 3 ? 3 : 2); ++r) {
    const V xr = r == 0 ? x0 : (r == 1 ? x1 : x2);
    V t = xr * V(-p.sfree);
    t = fmav(x0, V(p.s2h[r][0]), t);
    t = fmav(x1, V(p.s2h[r][1]), t);
    if constexpr (NZ == 3) t = fmav(x2, V(p.s2h[r][2]), t);
    En[r] = t;
  }
  if constexpr (NZ != 3) En[2] = V(0.0f);
  const V Exy = X[1][1][0] * V(p.soff[0] - p.sfree);
  const V Exz = NZ == 3 ? X[1][0][NZ - 2] * V(p.soff[1] - p.sfree) : V(0.0f);
  const V Eyz = NZ == 3 ? X[0][1][NZ - 2] * V(p.soff[2] - p.sfree) : V(0.0f);
  // per-axis entries of G
  V g1[3], g2[3], g21[3];
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    g1[al] = u[al];
    g21[al] = V(2.0f) * u[al];
    if constexpr (SH && HE) g2[al] = fmav(u[al], u[al], V(p.mu2[al]));
    else if constexpr (SH) g2[al] = u[al] * u[al];
    else g2[al] = V(p.mu2[al]);
  }
  // G[axis][a][a'] with the structural zeros and ones resolved at compile time
  auto coef = [&](int al, int a, int ap, bool& one, bool& zero) -> V {
    one = false; zero = false;
    if (a == ap) { one = true; return V(1.0f); }
    if (a < ap) { zero = true; return V(0.0f); }
    if (a - ap == 1) {
      if (!SH) { zero = true; return V(0.0f); }
      return a == 1 ? g1[al] : g21[al];
    }
    return g2[al];                                   // a = 2, a' = 0
  };
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c) {
        if (absent<LAT>(a, b, c) || a + b + c < 2) continue;
        const int cc = NZ == 3 ? c : 0;
        V acc = V(0.0f);
        bool any = false;
        // the six second-order sources (a', b', c')
#pragma unroll
        for (int sidx = 0; sidx < 6; ++sidx) {
          const int ap = sidx == 0 ? 2 : (sidx == 3 || sidx == 4 ? 1 : 0);
          const int bp = sidx == 1 ? 2 : (sidx == 3 || sidx == 5 ? 1 : 0);
          const int cp = sidx == 2 ? 2 : (sidx == 4 || sidx == 5 ? 1 : 0);
          if (NZ != 3 && cp != 0) continue;
          if (ap > a || bp > b || cp > cc) continue;
          bool o1, z1, o2, z2, o3, z3;
          const V fx = coef(0, a, ap, o1, z1), fy = coef(1, b, bp, o2, z2), fz = coef(2, cc, cp, o3, z3);
          if (z1 || z2 || z3) continue;
          const V src = sidx < 3 ? En[sidx] : (sidx == 3 ? Exy : (sidx == 4 ? Exz : Eyz));
          V term = src;
          if (!o1) term = term * fx;
          if (!o2) term = term * fy;
          if (!o3) term = term * fz;
          acc = any ? acc + term : term;
          any = true;
        }
        if (any) q.v[a][b][c] -= acc;
      }
}

// Collision of one node (or a pair of nodes, V = F2) in moment space,// Collision of one node (or a pair of nodes, V = F2) in moment space,
// Eq. (2-2-3):
//   m* - m0 = m(delta) + dt (m_G + m_F) - S (m^ne + dt m_F / 2),
// central variant: S replaced by N(u)^-1 Sbar N(u) (Eq. 5-1-2).
// bprev / bnow (simplified NCDE only): B(t - dt) / c of the node in, B(t) / c
// out; G = g^eq(0, (I - S_1/2) dB/dt, 0) of Eq. (4-16).
template <int LAT, int BASIS, bool FORCED, bool NSE, typename V, typename P>
__device__ __forceinline__ void collide(Cube<LAT, V>& q, const P& p, const V* bprev = nullptr, V* bnow = nullptr) {
  using S = PScalar<P>;
  constexpr int D = Lat<LAT>::D, NZ = Lat<LAT>::NZ;
  q.forward();
  V jh[3] = {q.v[1][0][0], q.v[0][1][0], V(0.0f)};
  if constexpr (NZ == 3) jh[2] = q.v[0][0][NZ - 2];
  const Macro<V> mc = macroscopic<D, NSE>(q.v[0][0][0], jh, p);

  // forcing moments (index units): F = g^eq(Sbar, Fbar, -c_s^2 Sbar I) (NSE)
  // or omega S (NCDE); G = g^eq(0, 0, M_2G), M_2G = (I - S_2/2)(u F + F u +
  // c_s^2 Sbar I) (NSE), or G = g^eq(0, (I - S_1/2) B' S, 0) (NCDE).
  V FA = V(0.0f), FB[3] = {V(0.0f), V(0.0f), V(0.0f)};
  V FM[6] = {V(0.0f), V(0.0f), V(0.0f), V(0.0f), V(0.0f), V(0.0f)};
  V GB[3] = {V(0.0f), V(0.0f), V(0.0f)}, GM[6] = {V(0.0f), V(0.0f), V(0.0f), V(0.0f), V(0.0f), V(0.0f)};
  if constexpr (FORCED) {
    FA = V(p.source);
    if constexpr (NSE) {
#pragma unroll
      for (int al = 0; al < 3; ++al) { FB[al] = V(p.fh[al]); FM[al] = V(-p.source * p.mu2[al]); }
      V Y[6];
#pragma unroll
      for (int al = 0; al < 3; ++al) Y[al] = fmav(mc.u[al], V(S(2) * p.fh[al]), V(p.source * p.mu2[al]));
      Y[3] = fmav(mc.u[0], V(p.fh[1]), mc.u[1] * V(p.fh[0]));
      Y[4] = fmav(mc.u[0], V(p.fh[2]), mc.u[2] * V(p.fh[0]));
      Y[5] = fmav(mc.u[1], V(p.fh[2]), mc.u[2] * V(p.fh[1]));
#pragma unroll
      for (int r = 0; r < D; ++r) {
        V t = Y[r];
#pragma unroll
        for (int k = 0; k < D; ++k) t = fmav(Y[k], V(S(-0.5) * p.s2h[r][k]), t);
        GM[r] = t;
      }
      GM[3] = Y[3] * V(S(1) - S(0.5) * p.soff[0]);
      GM[4] = Y[4] * V(S(1) - S(0.5) * p.soff[1]);
      GM[5] = Y[5] * V(S(1) - S(0.5) * p.soff[2]);
    } else if (p.kind >= KIND_NCDE_SIMPLE_LINEAR) {
      // first-order difference dB/dt = (B(t) - B(t - dt)) / dt; zero without a previous value
      const S idt = S(1) / p.dt;
#pragma unroll
      for (int al = 0; al < 3; ++al) {
        const V db = (bprev != nullptr && !p.hist_fresh) ? (mc.B[al] - bprev[al]) * V(idt) : V(0.0f);
        GB[al] = db * V(S(1) - S(0.5) * p.s1[al]);
        if (bnow != nullptr) bnow[al] = mc.B[al];
      }
    } else {
      const V bp = p.kind == KIND_NCDE_LINEAR ? V(1.0f) : mc.rho;   // B' = u bp
#pragma unroll
      for (int al = 0; al < 3; ++al) GB[al] = bp * V((S(1) - S(0.5) * p.s1[al]) * p.advh[al] * p.source);
    }
  }
  const V zero3[3] = {V(0.0f), V(0.0f), V(0.0f)};
  const V zero6[6] = {V(0.0f), V(0.0f), V(0.0f), V(0.0f), V(0.0f), V(0.0f)};
  const S hdt = S(0.5) * p.dt;

  // X = m^ne + dt m_F / 2 ; q becomes m(delta) + dt (m_G + m_F)
  V X[3][3][NZ];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c) {
        if (absent<LAT>(a, b, c)) { X[a][b][c] = V(0.0f); continue; }
        const V meq = meq_moment<LAT>(a, b, c, mc.dA, mc.B, mc.M, p);
        X[a][b][c] = q.v[a][b][c] - meq;
        if constexpr (FORCED) {
          const V mF = meq_moment<LAT>(a, b, c, FA, FB, FM, p);
          const V mG = NSE ? meq_moment<LAT>(a, b, c, V(0.0f), zero3, GM, p)
                           : meq_moment<LAT>(a, b, c, V(0.0f), GB, zero6, p);
          X[a][b][c] = fmav(mF, V(hdt), X[a][b][c]);
          q.v[a][b][c] = fmav(mG + mF, V(p.dt), q.v[a][b][c]);
        }
      }
  if constexpr (BASIS != 0 && NSE) {
    // raw step at the single rate s_free, then the transported correction
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c)
          if (!absent<LAT>(a, b, c) && a + b + c >= 2) q.v[a][b][c] = fmav(X[a][b][c], V(-p.sfree), q.v[a][b][c]);
    subtract_transported<LAT, BASIS>(q, X, mc.u, p);
  } else if constexpr (BASIS != 0) {
    Cube<LAT, V> k;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) k.v[a][b][c] = X[a][b][c];
    // Mbar = N M (Eq. 5-1-1): N = shift to central moments (bit 0 of
    // BASIS), then Hermite polynomials (bit 1)
    if constexpr ((BASIS & 1) != 0) k.template shift<false>(mc.u);
    if constexpr ((BASIS & 2) != 0) hermite_axes<false>(k, p);
    Cube<LAT, V> sk;
    relax<LAT, NSE, false>(sk.v, k.v, p);
    if constexpr ((BASIS & 2) != 0) hermite_axes<true>(sk, p);
    if constexpr ((BASIS & 1) != 0) sk.template shift<true>(mc.u);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) q.v[a][b][c] -= sk.v[a][b][c];
  } else {
    relax<LAT, NSE, true>(q.v, X, p);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < NZ; ++c)
        if (absent<LAT>(a, b, c)) q.v[a][b][c] = V(0.0f);
  q.inverse();
}

template <int LAT>
__device__ __forceinline__ constexpr int zi(int ez) { return Lat<LAT>::NZ == 3 ? ez + 1 : 0; }

// Storage scaling: FP16 and E3M12 populations are stored times a power of
// two near 1/omega_j (keeps small-weight deviations out of the subnormal
// range; E3M12 also carries its 2^(bias - 127) in the factor); BF16 has
// FP32's exponent range and, like 32/64-bit storage, is unscaled.
template <typename ST>
__device__ __forceinline__ constexpr bool scaled_storage() {
  return std::is_same<ST, __half>::value || std::is_same<ST, E3M12>::value;
}
template <typename ST>
__device__ __forceinline__ constexpr bool storage16() {
  return std::is_same<ST, __half>::value || std::is_same<ST, __nv_bfloat16>::value || std::is_same<ST, E3M12>::value;
}

// Two FP32 values to one word of two 16-bit codes (lo in the low half) with
// stochastic rounding: the discarded part of each value is compared with
// random bits, so the rounding error has mean zero and no correlation from
// one step to the next (round-to-nearest repeats the same error while a
// slowly varying population changes by less than a unit in the last place
// per step, and that error then grows with the step count).  FP16 and BF16
// use the conversion instruction with a random-bits operand (the low 16
// bits of r round lo, the high 16 bits round hi); E3M12 adds the random bits
// below its last place and truncates.
template <typename ST>
__device__ __forceinline__ unsigned sr_pack2(float lo, float hi, unsigned r) {
  if constexpr (std::is_same<ST, E3M12>::value) {
    return e3m12_encode2_sr(lo, hi, r);
  } else {
    unsigned d;
    if constexpr (std::is_same<ST, __half>::value)
      asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    else
      asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
  }
}

// The stores of the step kernels: 16-bit storage rounds stochastically,
// FP32 and FP64 store the value.
template <typename ST, typename CT>
__device__ __forceinline__ void store_step(ST* p, CT v, unsigned r) {
  if constexpr (storage16<ST>()) {
    const unsigned w = sr_pack2<ST>(float(v), 0.0f, r);
    *reinterpret_cast<unsigned short*>(p) = (unsigned short)(w & 0xFFFFu);
  } else {
    store_st<ST, CT>(p, v);
  }
}

// ------------------------------------------------------------------ kernels
// Coordinates of a step block's row: grid.y = y and grid.z = z, offset by
// p.plane0 along the slab axis (y on the 2-D lattices, z on the 3-D ones)
// when a launch covers only some of the planes (rmrtlb_step_interior /
// rmrtlb_step_boundary).
template <int LAT, typename P>
__device__ __forceinline__ int plane_y(const P& p) {
  return int(blockIdx.y) + (Lat<LAT>::D == 2 ? p.plane0 : 0);
}
template <int LAT, typename P>
__device__ __forceinline__ int plane_z(const P& p) {
  return int(blockIdx.z) + (Lat<LAT>::D == 3 ? p.plane0 : 0);
}

// One time step: pull gather from fin (post-collision of the previous step,
// x - e_j), collide, store the post-collision state of node x in fout.
template <int LAT, typename ST, typename CT, int BASIS, bool FORCED, bool NSE>
__global__ void __launch_bounds__(128) step_kernel(const ST* __restrict__ fin, ST* __restrict__ fout,
                                                   const KParams<CT> p) {
  using L = Lat<LAT>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = plane_y<LAT>(p), z = plane_z<LAT>(p);
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
    CT v = load_st<ST, CT>(fin + j * N + idx);
    if constexpr (scaled_storage<ST>()) v *= p.sinv[j];
    q.v[ex + 1][ey + 1][zi<LAT>(ez)] = v;
  });
  const size_t own = (size_t(z) * p.ny + y) * p.nx + x;
  if constexpr (FORCED && !NSE) {
    if (p.kind >= KIND_NCDE_SIMPLE_LINEAR) {
      CT bprev[3] = {CT(0), CT(0), CT(0)}, bnow[3];
#pragma unroll
      for (int al = 0; al < L::D; ++al) bprev[al] = p.hist[al * N + own];
      collide<LAT, BASIS, FORCED, NSE>(q, p, bprev, bnow);
#pragma unroll
      for (int al = 0; al < L::D; ++al) p.hist[al * N + own] = bnow[al];
    } else {
      collide<LAT, BASIS, FORCED, NSE>(q, p);
    }
  } else {
    collide<LAT, BASIS, FORCED, NSE>(q, p);
  }
  SrBits rng(p.seed, unsigned(own) + p.node_base);
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    CT v = q.v[ex + 1][ey + 1][zi<LAT>(ez)];
    if constexpr (scaled_storage<ST>()) v *= p.sc[j];
    store_step<ST, CT>(fout + j * N + own, v, rng.template word<j>());
  });
}

// ------------------------------------------------------------------ paired storage access
template <typename ST> struct Pair;
template <> struct Pair<double> { using T = double2; };
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<__half> { using T = __half2; };
template <> struct Pair<__nv_bfloat16> { using T = __nv_bfloat162; };
template <> struct Pair<E3M12> { using T = unsigned; };

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
template <>
__device__ __forceinline__ void load_pair<E3M12, float>(const E3M12* p, float& lo, float& hi) {
  const float2 v = e3m12_decode2(__ldg(reinterpret_cast<const unsigned*>(p)));
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
// loads to the last pair and store nothing.  With FP32 compute the pair is
// collided as one F2 value (packed FP32 arithmetic); FP64 collides the two
// nodes one after the other.
template <int LAT, typename ST, typename CT, int BASIS, bool FORCED, bool NSE>
__global__ void __launch_bounds__(128, Tuning<LAT, int(sizeof(ST)), BASIS != 0>::X2_MIN_BLOCKS)
    step_kernel_x2(const ST* __restrict__ fin, ST* __restrict__ fout, const KParams<CT> p) {
  using L = Lat<LAT>;
  constexpr bool PACKED = std::is_same<CT, float>::value;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int x0 = 2 * t;
  const bool active = x0 < p.nx;
  const int xc = active ? x0 : p.nx - 2;
  const int lane = threadIdx.x & 31;
  const int y = plane_y<LAT>(p), z = plane_z<LAT>(p);
  const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
  const bool fix_lo = lane == 0;                       // needs x0 - 1 from memory
  const bool fix_hi = lane == 31 || xc + 2 >= p.nx;    // needs x0 + 2 from memory
  const int d_lo = (xc == 0 ? p.nx - 1 : xc - 1) - xc; // offsets of x0 - 1, x0 + 2 from x0
  const int d_hi = (xc + 2 >= p.nx ? 0 : xc + 2) - xc;
  const size_t N = p.N;
  // 32-bit offsets of the source rows (y - e_y, z - e_z) plus x0 (N < 2^31)
  int roff[3][Lat<LAT>::NZ];
#pragma unroll
  for (int ey = -1; ey <= 1; ++ey)
#pragma unroll
    for (int ez = -1; ez <= 1; ++ez) {
      if (Lat<LAT>::NZ == 1 && ez != 0) continue;
      const int sy = Nbr::up(ey, ym, y, yp), sz = Nbr::up(ez, zm, z, zp);
      roff[ey + 1][zi<LAT>(ez)] = (sz * p.ny + sy) * p.nx + xc;
    }
  using V = typename std::conditional<PACKED, F2, CT>::type;
  Cube<LAT, V> qa, qb;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < L::NZ; ++c) { qa.v[a][b][c] = V(0.0f); qb.v[a][b][c] = V(0.0f); }
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    const ST* src = fin + j * N + roff[ey + 1][zi<LAT>(ez)];
    CT lo, hi, va, vb;
    load_pair<ST, CT>(src, lo, hi);
    if constexpr (ex == 0) {
      va = lo; vb = hi;
    } else if constexpr (ex == 1) {
      CT prev = __shfl_up_sync(0xffffffffu, hi, 1);
      if (fix_lo) prev = load_st<ST, CT>(src + d_lo);
      va = prev; vb = lo;
    } else {
      CT next = __shfl_down_sync(0xffffffffu, lo, 1);
      if (fix_hi) next = load_st<ST, CT>(src + d_hi);
      va = hi; vb = next;
    }
    if constexpr (PACKED) {
      if constexpr (scaled_storage<ST>()) qa.v[ex + 1][ey + 1][zi<LAT>(ez)] = V(va, vb) * V(p.sinv[j]);
      else qa.v[ex + 1][ey + 1][zi<LAT>(ez)] = V(va, vb);
    } else {
      if constexpr (scaled_storage<ST>()) { va *= p.sinv[j]; vb *= p.sinv[j]; }
      qa.v[ex + 1][ey + 1][zi<LAT>(ez)] = va;
      qb.v[ex + 1][ey + 1][zi<LAT>(ez)] = vb;
    }
  });
  collide<LAT, BASIS, FORCED, NSE>(qa, p);
  if constexpr (!PACKED) collide<LAT, BASIS, FORCED, NSE>(qb, p);
  if (!active) return;
  const int own = (z * p.ny + y) * p.nx + x0;
  SrBits rng(p.seed, unsigned(own) + p.node_base);
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    CT va, vb;
    if constexpr (PACKED) {
      F2 r = qa.v[ex + 1][ey + 1][zi<LAT>(ez)];
      if constexpr (scaled_storage<ST>()) r = r * V(p.sc[j]);
      va = r.v.x; vb = r.v.y;
    } else {
      va = qa.v[ex + 1][ey + 1][zi<LAT>(ez)];
      vb = qb.v[ex + 1][ey + 1][zi<LAT>(ez)];
      if constexpr (scaled_storage<ST>()) { va *= p.sc[j]; vb *= p.sc[j]; }
    }
    if constexpr (storage16<ST>())
      *reinterpret_cast<unsigned*>(fout + j * N + own) = sr_pack2<ST>(float(va), float(vb), rng.template word<j>());
    else
      store_pair<ST, CT>(fout + j * N + own, va, vb);
  });
}


// One time step, four x-adjacent nodes (x0 .. x0 + 3, x0 a multiple of 4)
// per thread, for 16-bit storage (rD2Q9, rD3Q19, rD3Q27; nx a multiple of
// 4): every population is one aligned 8-byte load of four values, which
// doubles the bytes per load and halves the loads, shuffles and index
// arithmetic per node against step_kernel_x2 (the 16-bit kernels were
// limited by memory-level parallelism and issue, not by DRAM).  The loaded
// codes stay packed, two 16-bit codes per 32-bit word: pair A holds nodes
// (x0, x0 + 1), pair B (x0 + 2, x0 + 3).  For e_x = +1 the thread needs
// x0 - 1: the last code of the lane below (warp shuffle of one word), lane 0
// loading it; for e_x = -1 it needs x0 + 4 from the lane above, the last
// lane of a warp or of a row loading it (periodic wrap); byte permutes
// assemble the shifted pairs.  Pair A is decoded, collided (packed FP32)
// and re-encoded into its words before pair B is decoded, so the packed
// codes of the other pair, not a second FP32 cube, are what stays live
// beside the collision.
template <typename ST>
__device__ __forceinline__ float2 decode2(unsigned w) {
  if constexpr (std::is_same<ST, __half>::value) {
    __half2 h;
    memcpy(&h, &w, 4);
    return __half22float2(h);
  } else if constexpr (std::is_same<ST, E3M12>::value) {
    return e3m12_decode2(w);
  } else {
    __nv_bfloat162 h;
    memcpy(&h, &w, 4);
    return __bfloat1622float2(h);
  }
}
__device__ __forceinline__ unsigned load_code(const void* p) {
  return __ldg(reinterpret_cast<const unsigned short*>(p));
}

template <int LAT, typename ST, int BASIS, bool FORCED, bool NSE>
__device__ __forceinline__ void collide_pair(unsigned (&w)[Lat<LAT>::Q], const KParams<float>& p, const SrBits& rng,
                                             int slot) {
  using L = Lat<LAT>;
  Cube<LAT, F2> q;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < L::NZ; ++c) q.v[a][b][c] = F2(0.0f);
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    F2 v(decode2<ST>(w[j]));
    if constexpr (scaled_storage<ST>()) v = v * F2(p.sinv[j]);
    q.v[ex + 1][ey + 1][zi<LAT>(ez)] = v;
  });
  collide<LAT, BASIS, FORCED, NSE>(q, p);
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    F2 v = q.v[ex + 1][ey + 1][zi<LAT>(ez)];
    if constexpr (scaled_storage<ST>()) v = v * F2(p.sc[j]);
    w[j] = sr_pack2<ST>(v.v.x, v.v.y, slot == 0 ? rng.template word<2 * j>() : rng.template word<2 * j + 1>());
  });
}

template <int LAT, typename ST, int BASIS, bool FORCED, bool NSE>
__global__ void __launch_bounds__(128, Tuning<LAT, 2, BASIS != 0>::X4_MIN_BLOCKS) step_kernel_x4(const ST* __restrict__ fin, ST* __restrict__ fout,
                                                      const KParams<float> p) {
  using L = Lat<LAT>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int x0 = 4 * t;
  const bool active = x0 < p.nx;
  const int xc = active ? x0 : p.nx - 4;
  const int lane = threadIdx.x & 31;
  const int y = plane_y<LAT>(p), z = plane_z<LAT>(p);
  const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
  const bool fix_lo = lane == 0;                       // needs x0 - 1 from memory
  const bool fix_hi = lane == 31 || xc + 4 >= p.nx;    // needs x0 + 4 from memory
  const int d_lo = (xc == 0 ? p.nx - 1 : xc - 1) - xc;
  const int d_hi = (xc + 4 >= p.nx ? 0 : xc + 4) - xc;
  const size_t N = p.N;
  int roff[3][Lat<LAT>::NZ];
#pragma unroll
  for (int ey = -1; ey <= 1; ++ey)
#pragma unroll
    for (int ez = -1; ez <= 1; ++ez) {
      if (Lat<LAT>::NZ == 1 && ez != 0) continue;
      const int sy = Nbr::up(ey, ym, y, yp), sz = Nbr::up(ez, zm, z, zp);
      roff[ey + 1][zi<LAT>(ez)] = (sz * p.ny + sy) * p.nx + xc;
    }
  unsigned wa[L::Q], wb[L::Q];
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    const ST* src = fin + j * N + roff[ey + 1][zi<LAT>(ez)];
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(src));   // codes x0 .. x0 + 3
    if constexpr (ex == 0) {
      wa[j] = w.x; wb[j] = w.y;
    } else if constexpr (ex == 1) {
      // (x0 - 1, x0), (x0 + 1, x0 + 2): the code below x0 sits in the high half of prev
      unsigned prev = __shfl_up_sync(0xffffffffu, w.y, 1);
      if (fix_lo) prev = load_code(src + d_lo) << 16;
      wa[j] = __byte_perm(prev, w.x, 0x5432);
      wb[j] = __byte_perm(w.x, w.y, 0x5432);
    } else {
      // (x0 + 1, x0 + 2), (x0 + 3, x0 + 4): the code above x0 + 3 sits in the low half of next
      unsigned next = __shfl_down_sync(0xffffffffu, w.x, 1);
      if (fix_hi) next = load_code(src + d_hi);
      wa[j] = __byte_perm(w.x, w.y, 0x5432);
      wb[j] = __byte_perm(w.y, next, 0x5432);
    }
  });
  const int own = (z * p.ny + y) * p.nx + xc;
  const SrBits rng(p.seed, unsigned(own) + p.node_base);
  collide_pair<LAT, ST, BASIS, FORCED, NSE>(wa, p, rng, 0);
  collide_pair<LAT, ST, BASIS, FORCED, NSE>(wb, p, rng, 1);
  if (!active) return;
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    *reinterpret_cast<uint2*>(fout + j * N + own) = make_uint2(wa[j], wb[j]);
  });
}

}  // namespace rmrt
