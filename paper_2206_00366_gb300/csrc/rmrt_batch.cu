// Batched lid-driven cavities on rD2Q9, rD3Q19 and rD3Q27 (raw or central
// moments): many independent rectangular domains (own size, spacing and
// viscosity) advanced together, one launch per step over a list of row
// tiles, with half-way bounce-back walls, a moving lid, a per-domain FP64
// residual check and retirement of converged or unstable domains.  Chunks of
// check_every steps plus their check are replayed as a CUDA graph.
//
// The paper has no boundaries and no batching; the collision of every node
// is the same Eq. (2-2-3) step as the single-domain kernels (shared code in
// rmrt_device.cuh).  Walls: a population whose source node x - e_j lies
// outside the domain is the node's own post-collision population in the
// opposite direction (half-way bounce-back); crossing the lid (the face
// beyond the last node of the last axis, moving along x with U) adds
// 2 omega_j rho0 (c_j . U) / c_s^2, the linear term of the REDF (Eq. 3-3).
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/rmrtlb.h"
#include "rmrt_device.cuh"
#include "rmrt_host.h"

namespace rmrt {

// Per-domain constants every step reads, copied to shared memory by each
// block: the collision constants of the shared derivation (weights of
// Sec. III, rates of Eq. 4-31, S_2 of Eq. 5-8-1; the KParams fields the
// collision reads, by the same names), the geometry, the lid terms.
template <typename CT>
struct CParams {
  int nx, ny, nz, kind, basis, pad_;
  unsigned long long N;
  CT rho0, cs2, dt, source;
  CT c[3], mu2[3];
  CT s0, s1[3], s2h[3][3], soff[3], sfree;
  CT fh[3], advh[3], q19h[3];
};
template <typename CT>
struct BParams {
  CParams<CT> k;
  unsigned long long off;   // element offset of the domain's population block
  unsigned long long uoff;  // element offset of its residual snapshot (d planes)
  CT lid[27];               // 2 omega_j rho0 c_x e_jx U / c_s^2: lid term of a population arriving from the lid
};
// Constants only the population set/get and the initialisation read (from
// global memory).
struct BCold {
  double wd[27];            // omega_j
  double rho0d;
  double ned[3];            // (c_a^2 - c_s^2) dt / s_sa: diagonal of Eq. (4-35) per unit rho and du_a/dx_a
  double neo[3];            // c_s^2 dt / s_ab (xy, xz, yz): off-diagonal of Eq. (4-35)
};

template <int LAT>
__host__ __device__ constexpr int opposite_dir(int j) {
  int r = 0;
  for (int k = 0; k < Lat<LAT>::Q; ++k)
    if (Lat<LAT>::EX[k] == -Lat<LAT>::EX[j] && Lat<LAT>::EY[k] == -Lat<LAT>::EY[j] &&
        Lat<LAT>::EZ[k] == -Lat<LAT>::EZ[j])
      r = k;
  return r;
}

// Copies a domain's parameter block into shared memory (block-uniform).
template <typename CT>
__device__ __forceinline__ void load_params(BParams<CT>& sp, const BParams<CT>* dom, int d) {
  constexpr int W = int(sizeof(BParams<CT>) / 4);
  const int* src = reinterpret_cast<const int*>(dom + d);
  int* dst = reinterpret_cast<int*>(&sp);
  for (int i = threadIdx.x; i < W; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

// A tile is (domain, first row, first x, width | rows << 16): `rows`
// consecutive rows (numbered z * ny + y) of `width` nodes from x.
__device__ __forceinline__ int tile_width(const int4& t) { return t.w & 0xffff; }
__device__ __forceinline__ int tile_rows(const int4& t) { return t.w >> 16; }

// A node inside its domain: index (x fastest, 32-bit: q N < 2^31 per
// domain), which neighbours x -/+ 1 along each axis lie inside the box, and
// whether the node sits in the layer under the lid.
struct NodeXYZ {
  int own;
  bool xm, xp, ym, yp, zm, zp;
  bool top;
};
template <int LAT, typename CT>
__device__ __forceinline__ NodeXYZ node_at(int x, int y, int z, const BParams<CT>& sp) {
  NodeXYZ r;
  const int nx = sp.k.nx, ny = sp.k.ny, nz = sp.k.nz;
  r.own = (z * ny + y) * nx + x;
  r.xm = x > 0; r.xp = x < nx - 1;
  r.ym = y > 0; r.yp = y < ny - 1;
  r.zm = z > 0; r.zp = z < nz - 1;
  r.top = Lat<LAT>::D == 2 ? y == ny - 1 : z == nz - 1;
  return r;
}

// True when a source coordinate lies beyond the lid: the face after the
// last node of the last axis (y on rD2Q9, z on the 3-D lattices).
template <int LAT>
__device__ __forceinline__ bool from_lid(int sy, int sz, int ny, int nz) {
  return Lat<LAT>::D == 2 ? sy >= ny : sz >= nz;
}

// Row r of a tile (rows numbered z * ny + y) as (y, z), advanced by one row
// with a carry.
struct RowYZ {
  int y, z;
  __device__ __forceinline__ RowYZ(int row, int ny) : y(row % ny), z(row / ny) {}
  __device__ __forceinline__ void next(int ny) {
    if (++y == ny) { y = 0; ++z; }
  }
};

// Population j arriving at a node: pulled from x - e_j inside the domain,
// else bounced back from the node itself (half-way bounce-back), with the
// lid term when x - e_j lies beyond the lid.
template <int LAT, typename CT, typename ST, int j>
__device__ __forceinline__ CT gather(const ST* __restrict__ base, const NodeXYZ& n, const BParams<CT>& sp) {
  constexpr int ex = Lat<LAT>::EX[j], ey = Lat<LAT>::EY[j], ez = Lat<LAT>::EZ[j];
  constexpr int jo = opposite_dir<LAT>(j);
  constexpr bool up_lid = Lat<LAT>::D == 2 ? ey < 0 : ez < 0;   // source one layer beyond the last
  const bool inside = (ex > 0 ? n.xm : (ex < 0 ? n.xp : true)) && (ey > 0 ? n.ym : (ey < 0 ? n.yp : true)) &&
                      (ez > 0 ? n.zm : (ez < 0 ? n.zp : true));
  const int N = int(sp.k.N), nx = sp.k.nx, nxy = sp.k.nx * sp.k.ny;
  const int idx = inside ? j * N + n.own - ex - ey * nx - ez * nxy : jo * N + n.own;
  CT v = CT(__ldg(base + idx));
  if (ex != 0 && up_lid && n.top) v += sp.lid[j];
  return v;
}

template <int LAT, int BASIS, typename ST, typename CT>
__global__ void __launch_bounds__(256) batch_step_kernel(const ST* __restrict__ fin, ST* __restrict__ fout,
                                                         const BParams<CT>* __restrict__ dom,
                                                         const int4* __restrict__ tiles,
                                                         const int* __restrict__ active) {
  using L = Lat<LAT>;
  const int4 t = tiles[blockIdx.x];  // (domain, row, x0, width)
  if (active[t.x] != 1) return;      // retired: its last state stays in buffer A
  __shared__ BParams<CT> sp;
  load_params(sp, dom, t.x);
  if (int(threadIdx.x) >= tile_width(t)) return;
  const ST* base = fin + sp.off;
  const int N = int(sp.k.N);
  const int rows = tile_rows(t), x = t.z + int(threadIdx.x);
  RowYZ yz(t.y, sp.k.ny);
  for (int r = 0; r < rows; ++r, yz.next(sp.k.ny)) {
    const NodeXYZ n = node_at<LAT>(x, yz.y, yz.z, sp);
    Cube<LAT, CT> q;
    if constexpr (LAT == LAT_D3Q19) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c) q.v[a][b][c] = CT(0);
    }
    static_for<L::Q>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
      q.v[ex + 1][ey + 1][zi<LAT>(ez)] = gather<LAT, CT, ST, j>(base, n, sp);
    });
    collide<LAT, BASIS, false, true>(q, sp.k);
    ST* out = fout + sp.off + n.own;
    static_for<L::Q>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
      out[j * N] = ST(q.v[ex + 1][ey + 1][zi<LAT>(ez)]);
    });
  }
}

// FP32 storage: two nodes per thread, x0 + i and x0 + i + h (h = half the
// tile width, rounded up), so that every load and store instruction of a
// warp stays contiguous; the pair is collided as one F2 value in packed FP32
// arithmetic (one instruction per operation for both nodes).  A thread
// whose second node lies past the tile's width collides its first node
// twice and stores it once.
template <int LAT, int BASIS>
__global__ void __launch_bounds__(128) batch_step_kernel_x2(const float* __restrict__ fin, float* __restrict__ fout,
                                                            const BParams<float>* __restrict__ dom,
                                                            const int4* __restrict__ tiles,
                                                            const int* __restrict__ active) {
  using L = Lat<LAT>;
  const int4 t = tiles[blockIdx.x];  // (domain, row, x0, width)
  if (active[t.x] != 1) return;      // retired: its last state stays in buffer A
  __shared__ BParams<float> sp;
  load_params(sp, dom, t.x);
  const int w = tile_width(t), h = (w + 1) / 2;
  const int i = int(threadIdx.x);
  if (i >= h) return;
  const bool has_b = i + h < w;
  const float* base = fin + sp.off;
  const int N = int(sp.k.N);
  const int rows = tile_rows(t), xa = t.z + i, xb = has_b ? xa + h : xa;
  RowYZ yz(t.y, sp.k.ny);
  for (int r = 0; r < rows; ++r, yz.next(sp.k.ny)) {
    const NodeXYZ na = node_at<LAT>(xa, yz.y, yz.z, sp);
    const NodeXYZ nb = node_at<LAT>(xb, yz.y, yz.z, sp);
    Cube<LAT, F2> q;
    if constexpr (LAT == LAT_D3Q19) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c) q.v[a][b][c] = F2(0.0f);
    }
    static_for<L::Q>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
      q.v[ex + 1][ey + 1][zi<LAT>(ez)] =
          F2(gather<LAT, float, float, j>(base, na, sp), gather<LAT, float, float, j>(base, nb, sp));
    });
    collide<LAT, BASIS, false, true>(q, sp.k);
    float* out = fout + sp.off;
    static_for<L::Q>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
      const F2 v = q.v[ex + 1][ey + 1][zi<LAT>(ez)];
      out[j * N + na.own] = v.v.x;
      if (has_b) out[j * N + nb.own] = v.v.y;
    });
  }
}

// Density and velocity of a node from its gathered populations.
template <int LAT, typename ST, typename CT>
__device__ __forceinline__ void node_fields(const ST* __restrict__ base, const NodeXYZ& n, const BParams<CT>& sp,
                                            CT& s0, double u[3]) {
  using L = Lat<LAT>;
  CT m1[3] = {CT(0), CT(0), CT(0)};
  s0 = CT(0);
  static_for<L::Q>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
    const CT v = gather<LAT, CT, ST, j>(base, n, sp);
    s0 += v;
    if (ex) m1[0] += CT(ex) * v;
    if (ey) m1[1] += CT(ey) * v;
    if (ez) m1[2] += CT(ez) * v;
  });
  const CT inv = CT(1) / (sp.k.rho0 + s0);
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = a < L::D ? double(m1[a] * sp.k.c[a] * inv) : 0.0;
}

// Per-tile FP64 sums for the residual ||u - u_prev|| / ||u||: [0] sum
// |u - u_prev|^2, [1] sum |u|^2, [2] sum (rho - rho0), [3] max |u|^2
// (infinite when a value is not finite).
template <int LAT, typename ST, typename CT>
__global__ void __launch_bounds__(256) batch_check_kernel(const ST* __restrict__ fin,
                                                          const BParams<CT>* __restrict__ dom,
                                                          const int4* __restrict__ tiles,
                                                          const int* __restrict__ active,
                                                          double* __restrict__ uprev, int use_prev,
                                                          double* __restrict__ partials) {
  using L = Lat<LAT>;
  constexpr int D = L::D;
  const int4 t = tiles[blockIdx.x];
  __shared__ double red[4][8];
  double acc[4] = {0, 0, 0, 0};
  if (active[t.x] == 1) {
    __shared__ BParams<CT> sp;
    load_params(sp, dom, t.x);
    if (int(threadIdx.x) < tile_width(t)) {
      const size_t N = sp.k.N;
      double* up = uprev + sp.uoff;
      RowYZ yz(t.y, sp.k.ny);
      for (int r = 0; r < tile_rows(t); ++r, yz.next(sp.k.ny)) {
        const NodeXYZ n = node_at<LAT>(t.z + int(threadIdx.x), yz.y, yz.z, sp);
        CT s0;
        double u[3];
        node_fields<LAT, ST, CT>(fin + sp.off, n, sp, s0, u);
        double du2 = 0.0, u2 = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const double dlt = u[a] - (use_prev ? up[a * N + n.own] : 0.0);
          up[a * N + n.own] = u[a];
          du2 += dlt * dlt;
          u2 += u[a] * u[a];
        }
        acc[0] += du2;
        acc[1] += u2;
        acc[2] += double(s0);
        acc[3] = fmax(acc[3], isfinite(u2) && isfinite(double(s0)) ? u2 : INFINITY);
      }
    }
  }
  // block reduction in a fixed order (blockDim is a multiple of 32, <= 256);
  // sums for [0..2], maximum for [3]
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v = __shfl_down_sync(0xffffffffu, acc[k], o);
      acc[k] = k < 3 ? acc[k] + v : fmax(acc[k], v);
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][warp] = acc[k];
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w)
      s = threadIdx.x < 3 ? s + red[threadIdx.x][w] : fmax(s, red[threadIdx.x][w]);
    partials[size_t(blockIdx.x) * 4 + threadIdx.x] = s;
  }
}

// rho and u (1 + d planes) of one domain, grid-stride over its nodes.
template <int LAT, typename ST, typename CT>
__global__ void batch_fields_kernel(const ST* __restrict__ fin, const BParams<CT>* __restrict__ dom, int d,
                                    double* __restrict__ fields) {
  __shared__ BParams<CT> sp;
  load_params(sp, dom, d);
  const size_t N = sp.k.N;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += size_t(gridDim.x) * blockDim.x) {
    const int row = int(i / sp.k.nx);
    const NodeXYZ n = node_at<LAT>(int(i % sp.k.nx), row % sp.k.ny, row / sp.k.ny, sp);
    CT s0;
    double u[3];
    node_fields<LAT, ST, CT>(fin + sp.off, n, sp, s0, u);
    fields[i] = double(sp.k.rho0 + s0);
#pragma unroll
    for (int a = 0; a < Lat<LAT>::D; ++a) fields[(1 + a) * N + i] = u[a];
  }
}

// One block per domain: fixed-order sum of its tiles' partials, residual,
// retirement.  status: [0] residual, [1] mass deviation.  active[d]: 1
// stepping, 0 converged (residual < tol), -1 unstable (a non-finite velocity
// or |u| >= c_s at the check).  conv[d] = index of the check that retired it.
__global__ void __launch_bounds__(256) batch_reduce_kernel(const double* __restrict__ partials,
                                                           const int* __restrict__ tile_begin,
                                                           int* __restrict__ active, double* __restrict__ status,
                                                           int* __restrict__ conv, const int* __restrict__ counters,
                                                           const double* __restrict__ cs2, double tol) {
  const int d = blockIdx.x;
  if (active[d] != 1) return;
  __shared__ double sm[4][256];
  double acc[4] = {0, 0, 0, 0};
  for (int i = tile_begin[d] + threadIdx.x; i < tile_begin[d + 1]; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] += partials[size_t(i) * 4 + k];
    acc[3] = fmax(acc[3], partials[size_t(i) * 4 + 3]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (int(threadIdx.x) < s) {
#pragma unroll
      for (int k = 0; k < 3; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
      sm[3][threadIdx.x] = fmax(sm[3][threadIdx.x], sm[3][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int checks = counters[0];
    const double res = checks > 0 && sm[1][0] > 0 ? sqrt(sm[0][0] / sm[1][0]) : -1.0;
    status[2 * d] = res;
    status[2 * d + 1] = sm[2][0];
    if (!(sm[3][0] < cs2[d])) {
      active[d] = -1;
      conv[d] = checks;
    } else if (checks > 0 && res >= 0 && res < tol) {
      active[d] = 0;
      conv[d] = checks;
    }
  }
}

// Rest state fbar = omega rho0 in pull storage: every stored deviation is 0
// except the slots of the layer under the lid that stream into it: they
// bounce back as the opposite direction jo and gain lid[jo] = -lid[j], so
// they hold lid[j].  grid (blocks, ndomains), grid-stride over the layer.
template <int LAT, typename ST, typename CT>
__global__ void batch_rest_kernel(ST* __restrict__ f, const BParams<CT>* __restrict__ dom) {
  using L = Lat<LAT>;
  const BParams<CT>& p = dom[blockIdx.y];
  const int nx = p.k.nx, ny = p.k.ny, nz = p.k.nz;
  const size_t layer = L::D == 2 ? size_t(nx) : size_t(nx) * ny;
  const size_t first = L::D == 2 ? size_t(ny - 1) * nx : size_t(nz - 1) * nx * ny;
  for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < layer; t += size_t(gridDim.x) * blockDim.x) {
    const size_t n = first + t;
    static_for<L::Q>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int ex = L::EX[j], up = L::D == 2 ? L::EY[j] : L::EZ[j];
      if (up == 1 && ex != 0) f[p.off + size_t(j) * p.k.N + n] = ST(p.lid[j]);
    });
  }
}

// counters[0]: number of completed checks (a check with counters[0] > 0 has a
// previous snapshot).
__global__ void batch_bump_kernel(int* counters) {
  if (threadIdx.x == 0 && blockIdx.x == 0) counters[0] += 1;
}

// Direction j's components and opposite, at run time.
template <int LAT>
__device__ __forceinline__ void dir_of(int j, int& ex, int& ey, int& ez, int& jo) {
  static_for<Lat<LAT>::Q>([&](auto J) {
    constexpr int k = decltype(J)::value;
    constexpr int cx = Lat<LAT>::EX[k], cy = Lat<LAT>::EY[k], cz = Lat<LAT>::EZ[k], ko = opposite_dir<LAT>(k);
    if (k == j) {
      ex = cx;
      ey = cy;
      ez = cz;
      jo = ko;
    }
  });
}

// Canonical populations of one domain <-> storage, plane j.
// to_storage: plane = fbar_j (first N values) and fbar_jo (next N); slot
// A_j(x) = fbar_j(x + e_j) inside, else fbar_jo(x) - lid[jo] (the value that
// bounces back into jo).  from_storage: plane = fbar_j = gather.
template <int LAT, typename ST, typename CT>
__global__ void batch_plane_kernel(ST* __restrict__ f, double* __restrict__ plane, int j, int to_storage,
                                   const BParams<CT>* __restrict__ dom, const BCold* __restrict__ cold, int d) {
  __shared__ BParams<CT> sp;
  load_params(sp, dom, d);
  const int nx = sp.k.nx, ny = sp.k.ny, nz = sp.k.nz;
  const size_t N = sp.k.N;
  ST* base = f + sp.off;   // storage holds fbar - omega rho0 (omega_j = omega_opp(j))
  int ex = 0, ey = 0, ez = 0, jo = 0;
  dir_of<LAT>(j, ex, ey, ez, jo);
  const double rest = cold[d].wd[j] * cold[d].rho0d;
  for (size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x; n < N; n += size_t(gridDim.x) * blockDim.x) {
    const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (size_t(nx) * ny));
    if (to_storage) {
      const int tx = x + ex, ty = y + ey, tz = z + ez;
      double v;
      if (unsigned(tx) < unsigned(nx) && unsigned(ty) < unsigned(ny) && unsigned(tz) < unsigned(nz)) {
        v = plane[(size_t(tz) * ny + ty) * nx + tx];
      } else {
        v = plane[N + n];
        if (ex != 0 && from_lid<LAT>(ty, tz, ny, nz)) v -= double(sp.lid[jo]);
      }
      base[size_t(j) * N + n] = ST(v - rest);
    } else {
      const int sx = x - ex, sy = y - ey, sz = z - ez;
      double v;
      if (unsigned(sx) < unsigned(nx) && unsigned(sy) < unsigned(ny) && unsigned(sz) < unsigned(nz)) {
        v = double(base[size_t(j) * N + (size_t(sz) * ny + sy) * nx + sx]);
      } else {
        v = double(base[size_t(jo) * N + n]);
        if (ex != 0 && from_lid<LAT>(sy, sz, ny, nz)) v += double(sp.lid[j]);
      }
      plane[n] = v + rest;
    }
  }
}

// d u_b / d x_a at a node from a field (b-th plane of u): central difference
// inside, one-sided at the first and last node, 0 on a one-node axis.
__device__ __forceinline__ double grad_at(const double* __restrict__ ub, size_t n, int i, int len, size_t stride,
                                          double h) {
  if (len < 2) return 0.0;
  if (i == 0) return (ub[n + stride] - ub[n]) / h;
  if (i == len - 1) return (ub[n] - ub[n - stride]) / h;
  return (ub[n + stride] - ub[n - stride]) / (2.0 * h);
}

// fbar = f^eq(rho, u) (Eq. NSEfeq), plus with_ne the non-equilibrium part
// f^ne = g^eq(0, 0, m_2^ne) of Eq. (fne) with m_2^ne from Eq. (4-35):
// m_2^ne_aa = -rho (c_a^2 - c_s^2) dt du_a/dx_a / s_sa and
// m_2^ne_ab = -rho c_s^2 dt (du_a/dx_b + du_b/dx_a) / s_ab (a != b); both
// are the equilibrium moments of g^eq(rho, rho u, rho u u + m_2^ne).  Each
// value goes to the slot the next pull gather reads it from.
template <int LAT, typename ST, typename CT>
__global__ void batch_init_kernel(ST* __restrict__ f, const double* __restrict__ rho, const double* __restrict__ u,
                                  const BParams<CT>* __restrict__ dom, const BCold* __restrict__ cold, int d,
                                  int with_ne) {
  using L = Lat<LAT>;
  constexpr int D = L::D, NZ = L::NZ;
  __shared__ BParams<CT> sp;
  load_params(sp, dom, d);
  const CParams<CT>& p = sp.k;
  const BCold& cd = cold[d];
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const size_t N = p.N;
  ST* base = f + sp.off;
  for (size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x; n < N; n += size_t(gridDim.x) * blockDim.x) {
    const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (size_t(nx) * ny));
    const double r = rho[n];
    CT uh[3] = {CT(0), CT(0), CT(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) uh[a] = CT(u[a * N + n] / double(p.c[a]));
    Macro<CT> mc;
    mc.dA = CT(r - cd.rho0d);
    mc.rho = CT(r);
    // g^eq(rho, rho u, rho u u) of the NSE in index units (Eq. NSEfeq)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mc.u[a] = uh[a];
      mc.B[a] = CT(r) * uh[a];
    }
    mc.M[0] = CT(r) * uh[0] * uh[0]; mc.M[1] = CT(r) * uh[1] * uh[1]; mc.M[2] = CT(r) * uh[2] * uh[2];
    mc.M[3] = CT(r) * uh[0] * uh[1]; mc.M[4] = CT(r) * uh[0] * uh[2]; mc.M[5] = CT(r) * uh[1] * uh[2];
    if (with_ne) {
      const int idx[3] = {x, y, z}, len[3] = {nx, ny, nz};
      const size_t stride[3] = {1, size_t(nx), size_t(nx) * ny};
      double g[3][3];   // g[a][b] = d u_b / d x_a
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          g[a][b] = (a < D && b < D) ? grad_at(u + b * N, n, idx[a], len[a], stride[a], double(p.c[a]) * double(p.dt))
                                     : 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const double ca = double(p.c[a]);
        mc.M[a] += CT(-r * cd.ned[a] * g[a][a] / (ca * ca));
      }
      const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int a = pa[k], b = pb[k];
        if (a < D && b < D)
          mc.M[3 + k] += CT(-r * cd.neo[k] * (g[a][b] + g[b][a]) / (double(p.c[a]) * double(p.c[b])));
      }
    }
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
      constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j], jo = opposite_dir<LAT>(j);
      const CT v = q.v[ex + 1][ey + 1][zi<LAT>(ez)];
      const int sx = x - ex, sy = y - ey, sz = z - ez;
      if (unsigned(sx) < unsigned(nx) && unsigned(sy) < unsigned(ny) && unsigned(sz) < unsigned(nz)) {
        base[size_t(j) * N + (size_t(sz) * ny + sy) * nx + sx] = ST(v);
      } else {
        const CT lidj = (ex != 0 && from_lid<LAT>(sy, sz, ny, nz)) ? sp.lid[j] : CT(0);
        base[size_t(jo) * N + n] = ST(v - lidj);
      }
    });
  }
}

}  // namespace rmrt

using namespace rmrt;
using namespace rmrt::host;

namespace {

constexpr size_t kAlignB = 256;
size_t align_b(size_t v) { return (v + kAlignB - 1) / kAlignB * kAlignB; }
const int kWidths[4] = {32, 64, 128, 256};
const int kRows[3] = {1, 2, 4};

size_t nodes_of(const rmrtlb_domain& x) { return size_t(x.nx) * x.ny * x.nz; }
size_t rows_of(const rmrtlb_domain& x) { return size_t(x.ny) * x.nz; }

struct BatchLayout {
  size_t fA, fB, uprev, dom, cold, tiles, partials, tile_begin, active, status, conv, counters, cs2, stage, total;
  size_t pop_elems;          // elements of one population lattice (all domains)
  size_t max_tiles;
  size_t max_n;              // largest domain
};

size_t tiles_of(const rmrtlb_domain& x, int width, int rows) {
  return size_t((x.nx + width - 1) / width) * ((rows_of(x) + rows - 1) / rows);
}
size_t tiles_for(const std::vector<rmrtlb_domain>& d, int width, int rows) {
  size_t t = 0;
  for (const auto& x : d) t += tiles_of(x, width, rows);
  return t;
}

BatchLayout batch_layout(int lat, const std::vector<rmrtlb_domain>& d, int storage) {
  BatchLayout L;
  const int q = lattice_q(lat), dim = lattice_d(lat);
  const size_t es = storage == RMRTLB_ST_F64 ? 8 : 4;
  size_t elems = 0, unodes = 0, maxn = 0;
  for (const auto& x : d) {
    const size_t n = nodes_of(x);
    elems += align_b(q * n * es) / es;
    unodes += dim * n;
    maxn = n > maxn ? n : maxn;
  }
  L.pop_elems = elems;
  L.max_n = maxn;
  L.max_tiles = tiles_for(d, kWidths[0], 1);
  const size_t nd = d.size();
  const size_t psize = storage == RMRTLB_ST_F64 ? sizeof(BParams<double>) : sizeof(BParams<float>);
  L.fA = 0;
  L.fB = L.fA + align_b(elems * es);
  L.uprev = L.fB + align_b(elems * es);
  L.dom = L.uprev + align_b(unodes * sizeof(double));
  L.cold = L.dom + align_b(nd * psize);
  L.tiles = L.cold + align_b(nd * sizeof(BCold));
  L.partials = L.tiles + align_b(L.max_tiles * sizeof(int4));
  L.tile_begin = L.partials + align_b(L.max_tiles * 4 * sizeof(double));
  L.active = L.tile_begin + align_b((nd + 1) * sizeof(int));
  L.status = L.active + align_b(nd * sizeof(int));
  L.conv = L.status + align_b(2 * nd * sizeof(double));
  L.counters = L.conv + align_b(nd * sizeof(int));
  L.cs2 = L.counters + align_b(16 * sizeof(int));
  L.stage = L.cs2 + align_b(nd * sizeof(double));
  L.total = L.stage + align_b(size_t(dim + 1) * maxn * sizeof(double));
  return L;
}

bool domain_ok(int lat, const rmrtlb_domain& x) {
  if (x.nx < 1 || x.ny < 1 || x.nz < 1) return false;
  if (lat == RMRTLB_D2Q9 && x.nz != 1) return false;
  const double n = double(x.nx) * x.ny * x.nz;
  return n <= 2.0e9 / lattice_q(lat) && double(x.ny) * x.nz < 2.0e9;
}

// Parameters of one cavity from the same derivation as rmrtlb_create, plus
// the lid terms and the Eq. (4-35) coefficients.
template <typename CT>
int domain_params(int lat, int basis, int storage, const rmrtlb_domain& D, double rho0, BParams<CT>& p, BCold& cold,
                  double* cs2_out) {
  memset(&p, 0, sizeof(p));
  memset(&cold, 0, sizeof(cold));
  if (!domain_ok(lat, D) || !(D.nu > 0) || !(D.nu_bulk > 0)) return RMRTLB_EINVAL;
  rmrtlb_params rp;
  memset(&rp, 0, sizeof(rp));
  rp.cs2 = D.cs2;
  rp.rho0 = rho0;
  rp.nu = D.nu;
  rp.nu_bulk = D.nu_bulk;
  rp.s_free = D.s_free;
  Consts k;
  const int rc = make_consts(k, lat, D.nx, D.ny, D.nz, D.dx, D.dy, lat == RMRTLB_D2Q9 ? 1.0 : D.dz, 1.0, rp,
                             RMRTLB_EQ_NSE, basis, storage);
  if (rc) return rc;
  const KParams<CT> kp = to_kparams<CT>(k);
  CParams<CT>& c = p.k;
  c.nx = kp.nx; c.ny = kp.ny; c.nz = kp.nz; c.kind = kp.kind; c.basis = kp.basis;
  c.N = kp.N;
  c.rho0 = kp.rho0; c.cs2 = kp.cs2; c.dt = kp.dt; c.source = kp.source;
  for (int a = 0; a < 3; ++a) {
    c.c[a] = kp.c[a]; c.mu2[a] = kp.mu2[a]; c.s1[a] = kp.s1[a]; c.soff[a] = kp.soff[a];
    c.fh[a] = kp.fh[a]; c.advh[a] = kp.advh[a]; c.q19h[a] = kp.q19h[a];
    for (int b = 0; b < 3; ++b) c.s2h[a][b] = kp.s2h[a][b];
  }
  c.s0 = kp.s0; c.sfree = kp.sfree;
  for (int j = 0; j < k.q; ++j) {
    int e[3];
    lattice_dir(lat, j, e);
    p.lid[j] = CT(2.0 * k.w[j] * rho0 * k.c[0] * e[0] * D.lid_u / k.cs2);
    cold.wd[j] = k.w[j];
  }
  cold.rho0d = rho0;
  for (int a = 0; a < 3; ++a) {
    cold.ned[a] = a < k.d ? (k.c[a] * k.c[a] - k.cs2) * k.dt / k.ss[a] : 0.0;
    cold.neo[a] = k.cs2 * k.dt / k.soff[a];
  }
  *cs2_out = k.cs2;
  return RMRTLB_OK;
}

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct rmrtlb_batch {
  int lat, q, d, central;
  std::vector<rmrtlb_domain> dom;
  std::vector<int> tile_begin_host;
  BatchLayout L;
  int storage;
  char* ws;
  cudaStream_t stream;
  int width;                        // tile width (nodes)
  int rows;                         // rows per tile
  int per_thread;                   // nodes per thread: 1, 2 (FP32, packed) or 0 (automatic, FP32)
  size_t live_nodes;                // nodes of the domains in the tile list
  size_t fill_nodes;                // twice the GPU's resident threads
  size_t ntiles;
  int check_every;
  double tol;
  long long step;
  int cur;                          // 0: state in A
  std::vector<long long> check_steps;
  cudaGraphExec_t graph;
  bool graph_ok;
};

namespace {

template <typename T> T* at(rmrtlb_batch* b, size_t off) { return reinterpret_cast<T*>(b->ws + off); }

// Row tiles of every domain (act == NULL) or of the domains still stepping
// (act[d] == 1); tile_begin[d] .. tile_begin[d + 1] are domain d's tiles
// (an empty range for a domain left out).
cudaError_t build_tiles(rmrtlb_batch* b, int width, int rows, const std::vector<int>* act = nullptr) {
  std::vector<int4> t;
  std::vector<int> tb(b->dom.size() + 1, 0);
  size_t live = 0;
  for (size_t d = 0; d < b->dom.size(); ++d) {
    tb[d] = int(t.size());
    if (act && (*act)[d] != 1) continue;
    const auto& D = b->dom[d];
    live += nodes_of(D);
    const int nr = int(rows_of(D));
    for (int r = 0; r < nr; r += rows)
      for (int x0 = 0; x0 < D.nx; x0 += width) {
        const int w = D.nx - x0 < width ? D.nx - x0 : width;
        const int h = nr - r < rows ? nr - r : rows;
        t.push_back(make_int4(int(d), r, x0, w | (h << 16)));
      }
  }
  tb[b->dom.size()] = int(t.size());
  b->ntiles = t.size();
  b->live_nodes = live;
  b->width = width;
  b->rows = rows;
  b->tile_begin_host = tb;
  if (t.empty()) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(at<int4>(b, b->L.tiles), t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                  b->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(at<int>(b, b->L.tile_begin), tb.data(), tb.size() * sizeof(int), cudaMemcpyHostToDevice,
                      b->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(b->stream);   // host vectors go out of scope
}

void drop_graph(rmrtlb_batch* b) {
  if (b->graph_ok) cudaGraphExecDestroy(b->graph);
  b->graph_ok = false;
}

// Two nodes per thread (packed FP32) when asked for, or, in the automatic
// mode, while the domains being stepped hold at least twice as many nodes
// as the GPU has resident threads; below that a thread per node finishes a
// step sooner (the tail of a batch run, small batches).
bool pairs(const rmrtlb_batch* b) {
  return b->per_thread == 2 || (b->per_thread == 0 && b->live_nodes >= b->fill_nodes);
}

// Kernel launches, one functor per kernel; dispatch() picks the template
// instance for the batch's lattice, basis and storage.
struct StepF {
  rmrtlb_batch* b;
  template <int LAT, int BASIS, typename ST, typename CT>
  cudaError_t run() const {
    if (b->ntiles == 0) return cudaSuccess;
    const ST* fin = at<ST>(b, b->cur == 0 ? b->L.fA : b->L.fB);
    ST* fout = at<ST>(b, b->cur == 0 ? b->L.fB : b->L.fA);
    if constexpr (std::is_same<ST, float>::value) {
      if (pairs(b)) {
        batch_step_kernel_x2<LAT, BASIS><<<unsigned(b->ntiles), (b->width + 1) / 2, 0, b->stream>>>(
            fin, fout, at<BParams<CT>>(b, b->L.dom), at<int4>(b, b->L.tiles), at<int>(b, b->L.active));
      } else {
        batch_step_kernel<LAT, BASIS, ST, CT><<<unsigned(b->ntiles), b->width, 0, b->stream>>>(
            fin, fout, at<BParams<CT>>(b, b->L.dom), at<int4>(b, b->L.tiles), at<int>(b, b->L.active));
      }
    } else {
      batch_step_kernel<LAT, BASIS, ST, CT><<<unsigned(b->ntiles), b->width, 0, b->stream>>>(
          fin, fout, at<BParams<CT>>(b, b->L.dom), at<int4>(b, b->L.tiles), at<int>(b, b->L.active));
    }
    return cudaGetLastError();
  }
};
struct CheckF {
  rmrtlb_batch* b;
  template <int LAT, int BASIS, typename ST, typename CT>
  cudaError_t run() const {
    if (b->ntiles == 0) return cudaSuccess;
    const ST* fin = at<ST>(b, b->cur == 0 ? b->L.fA : b->L.fB);
    batch_check_kernel<LAT, ST, CT><<<unsigned(b->ntiles), b->width, 0, b->stream>>>(
        fin, at<BParams<CT>>(b, b->L.dom), at<int4>(b, b->L.tiles), at<int>(b, b->L.active),
        at<double>(b, b->L.uprev), 1, at<double>(b, b->L.partials));
    return cudaGetLastError();
  }
};
struct FieldsF {
  rmrtlb_batch* b;
  int which, domain;
  double* fields;
  template <int LAT, int BASIS, typename ST, typename CT>
  cudaError_t run() const {
    const size_t N = nodes_of(b->dom[domain]);
    const unsigned grid = unsigned(N / 256 + 1 < 4096 ? N / 256 + 1 : 4096);
    batch_fields_kernel<LAT, ST, CT><<<grid, 256, 0, b->stream>>>(at<ST>(b, which == 0 ? b->L.fA : b->L.fB),
                                                                 at<BParams<CT>>(b, b->L.dom), domain, fields);
    return cudaGetLastError();
  }
};
struct RestF {
  rmrtlb_batch* b;
  template <int LAT, int BASIS, typename ST, typename CT>
  cudaError_t run() const {
    int maxlayer = 1;
    for (const auto& d : b->dom) {
      const int l = LAT == LAT_D2Q9 ? d.nx : d.nx * d.ny;
      maxlayer = l > maxlayer ? l : maxlayer;
    }
    const int bx = (maxlayer + 127) / 128 < 64 ? (maxlayer + 127) / 128 : 64;
    batch_rest_kernel<LAT, ST, CT><<<dim3(unsigned(bx), unsigned(b->dom.size())), 128, 0, b->stream>>>(
        at<ST>(b, b->L.fA), at<BParams<CT>>(b, b->L.dom));
    return cudaGetLastError();
  }
};
struct PlaneF {
  rmrtlb_batch* b;
  int which;
  double* pl;
  int j, to_storage, domain;
  template <int LAT, int BASIS, typename ST, typename CT>
  cudaError_t run() const {
    const size_t N = nodes_of(b->dom[domain]);
    const unsigned grid = unsigned(N / 256 + 1 < 4096 ? N / 256 + 1 : 4096);
    batch_plane_kernel<LAT, ST, CT><<<grid, 256, 0, b->stream>>>(at<ST>(b, which == 0 ? b->L.fA : b->L.fB), pl, j,
                                                                to_storage, at<BParams<CT>>(b, b->L.dom),
                                                                at<BCold>(b, b->L.cold), domain);
    return cudaGetLastError();
  }
};
struct InitF {
  rmrtlb_batch* b;
  int which;
  const double* rho;
  const double* u;
  int domain, with_ne;
  template <int LAT, int BASIS, typename ST, typename CT>
  cudaError_t run() const {
    const size_t N = nodes_of(b->dom[domain]);
    const unsigned grid = unsigned(N / 128 + 1 < 8192 ? N / 128 + 1 : 8192);
    batch_init_kernel<LAT, ST, CT><<<grid, 128, 0, b->stream>>>(at<ST>(b, which == 0 ? b->L.fA : b->L.fB), rho, u,
                                                               at<BParams<CT>>(b, b->L.dom), at<BCold>(b, b->L.cold),
                                                               domain, with_ne);
    return cudaGetLastError();
  }
};

template <int LAT, int BASIS, typename F>
cudaError_t dispatch_st(rmrtlb_batch* b, const F& f) {
  return b->storage == RMRTLB_ST_F64 ? f.template run<LAT, BASIS, double, double>()
                                     : f.template run<LAT, BASIS, float, float>();
}
template <int LAT, typename F>
cudaError_t dispatch_basis(rmrtlb_batch* b, const F& f) {
  switch (b->central) {
    case 1: return dispatch_st<LAT, 1>(b, f);
    case 2: return dispatch_st<LAT, 2>(b, f);
    case 3: return dispatch_st<LAT, 3>(b, f);
    default: return dispatch_st<LAT, 0>(b, f);
  }
}
template <typename F>
cudaError_t dispatch(rmrtlb_batch* b, const F& f) {
  switch (b->lat) {
    case RMRTLB_D3Q19: return dispatch_basis<LAT_D3Q19>(b, f);
    case RMRTLB_D3Q27: return dispatch_basis<LAT_D3Q27>(b, f);
    default: return dispatch_basis<LAT_D2Q9>(b, f);
  }
}

cudaError_t do_step(rmrtlb_batch* b) {
  return dispatch(b, StepF{b});
}

cudaError_t do_check(rmrtlb_batch* b) {
  cudaError_t e = dispatch(b, CheckF{b});
  if (e != cudaSuccess) return e;
  batch_reduce_kernel<<<unsigned(b->dom.size()), 256, 0, b->stream>>>(
      at<double>(b, b->L.partials), at<int>(b, b->L.tile_begin), at<int>(b, b->L.active),
      at<double>(b, b->L.status), at<int>(b, b->L.conv), at<int>(b, b->L.counters), at<double>(b, b->L.cs2), b->tol);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_bump_kernel<<<1, 32, 0, b->stream>>>(at<int>(b, b->L.counters));
  return cudaGetLastError();
}

// One chunk: check_every steps (even, so the state ends in A again) and the check.
cudaError_t chunk_direct(rmrtlb_batch* b) {
  for (int i = 0; i < b->check_every; ++i) {
    cudaError_t e = do_step(b);
    if (e != cudaSuccess) return e;
    b->cur ^= 1;
  }
  return do_check(b);
}

cudaError_t chunk(rmrtlb_batch* b) {
  if (b->stream == nullptr) return chunk_direct(b);
  if (!b->graph_ok) {
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const int cur0 = b->cur;
    e = chunk_direct(b);
    b->cur = cur0;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) return e;
    if (e2 != cudaSuccess) return e2;
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    b->graph_ok = true;
  }
  return cudaGraphLaunch(b->graph, b->stream);   // chunk_direct's parity changes cancel: check_every is even
}

cudaError_t reset_state(rmrtlb_batch* b) {
  const size_t es = b->storage == RMRTLB_ST_F64 ? 8 : 4;
  if (b->ntiles != tiles_for(b->dom, b->width, b->rows)) {   // a compacted list: every domain steps again
    drop_graph(b);
    cudaError_t e = build_tiles(b, b->width, b->rows);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemsetAsync(b->ws + b->L.fA, 0, b->L.pop_elems * es, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.fB, 0, b->L.pop_elems * es, b->stream);
  if (e == cudaSuccess) e = dispatch(b, RestF{b});
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.uprev, 0, b->L.dom - b->L.uprev, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.counters, 0, 16 * sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.status, 0, 2 * b->dom.size() * sizeof(double), b->stream);
  std::vector<int> one(b->dom.size(), 1), neg(b->dom.size(), -1);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(at<int>(b, b->L.active), one.data(), one.size() * sizeof(int), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(at<int>(b, b->L.conv), neg.data(), neg.size() * sizeof(int), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  b->step = 0;
  b->cur = 0;
  b->check_steps.clear();
  return e;
}

// Current buffer of a domain: a retired domain's state stays in A.
int domain_buffer(rmrtlb_batch* b, int domain, int* which) {
  int act = 1;
  if (cudaMemcpyAsync(&act, b->ws + b->L.active + domain * sizeof(int), sizeof(int), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  *which = act == 1 ? b->cur : 0;
  return RMRTLB_OK;
}

// State flags of every domain (synchronises).
int read_active(rmrtlb_batch* b, std::vector<int>& act) {
  act.resize(b->dom.size());
  if (cudaMemcpyAsync(act.data(), b->ws + b->L.active, act.size() * sizeof(int), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

}  // namespace

extern "C" {

int rmrtlb_batch_workspace_bytes(int lattice, int ndomains, const rmrtlb_domain* domains, int storage,
                                 size_t* bytes) {
  if (lattice < 0 || lattice > 2 || ndomains < 1 || ndomains > 65535 || !domains || !bytes ||
      (storage != RMRTLB_ST_F32 && storage != RMRTLB_ST_F64))
    return RMRTLB_EINVAL;
  std::vector<rmrtlb_domain> d(domains, domains + ndomains);
  for (const auto& x : d)
    if (!domain_ok(lattice, x)) return RMRTLB_EINVAL;
  if (tiles_for(d, kWidths[0], 1) > size_t(1) << 31) return RMRTLB_EINVAL;
  *bytes = batch_layout(lattice, d, storage).total;
  return RMRTLB_OK;
}

int rmrtlb_batch_create(rmrtlb_batch_t* out, int lattice, int basis, int ndomains, const rmrtlb_domain* domains,
                        int storage, double rho0, int check_every, double tol, void* workspace,
                        size_t workspace_bytes, void* stream) {
  if (!out) return RMRTLB_EINVAL;
  *out = nullptr;
  size_t need = 0;
  int rc = rmrtlb_batch_workspace_bytes(lattice, ndomains, domains, storage, &need);
  if (rc) return rc;
  if (basis < 0 || basis > 3) return RMRTLB_EINVAL;
  if (!workspace || reinterpret_cast<size_t>(workspace) % kAlignB) return RMRTLB_EINVAL;
  if (workspace_bytes < need) return RMRTLB_ENOMEM;
  if (check_every < 2 || !(tol > 0) || !isfinite(rho0)) return RMRTLB_EINVAL;
  rmrtlb_batch* b = new (std::nothrow) rmrtlb_batch();
  if (!b) return RMRTLB_ENOMEM;
  b->lat = lattice;
  b->q = lattice_q(lattice);
  b->d = lattice_d(lattice);
  b->central = basis;
  b->dom.assign(domains, domains + ndomains);
  for (auto& x : b->dom)
    if (lattice == RMRTLB_D2Q9) x.dz = 1.0;
  b->storage = storage;
  b->L = batch_layout(lattice, b->dom, storage);
  b->ws = static_cast<char*>(workspace);
  b->stream = static_cast<cudaStream_t>(stream);
  b->check_every = check_every + (check_every & 1);
  b->tol = tol;
  b->graph_ok = false;
  // parameter blocks and population offsets
  const size_t es = storage == RMRTLB_ST_F64 ? 8 : 4;
  size_t off = 0, uoff = 0;
  const size_t psize = storage == RMRTLB_ST_F64 ? sizeof(BParams<double>) : sizeof(BParams<float>);
  std::vector<char> params(ndomains * psize);
  std::vector<BCold> cold(ndomains);
  std::vector<double> cs2(ndomains);
  for (int d = 0; d < ndomains; ++d) {
    const size_t n = nodes_of(b->dom[d]);
    if (storage == RMRTLB_ST_F64) {
      BParams<double> p;
      rc = domain_params(lattice, basis, storage, b->dom[d], rho0, p, cold[d], &cs2[d]);
      p.off = off; p.uoff = uoff;
      memcpy(params.data() + d * psize, &p, psize);
    } else {
      BParams<float> p;
      rc = domain_params(lattice, basis, storage, b->dom[d], rho0, p, cold[d], &cs2[d]);
      p.off = off; p.uoff = uoff;
      memcpy(params.data() + d * psize, &p, psize);
    }
    if (rc) { delete b; return rc; }
    off += align_b(b->q * n * es) / es;
    uoff += b->d * n;
  }
  cudaError_t e = cudaMemcpyAsync(b->ws + b->L.dom, params.data(), params.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + b->L.cs2, cs2.data(), cs2.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + b->L.cold, cold.data(), cold.size() * sizeof(BCold), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  b->rows = 1;
  b->per_thread = storage == RMRTLB_ST_F32 ? 0 : 1;
  {
    int dev = 0, sms = 0, tps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&tps, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    b->fill_nodes = 2 * size_t(sms) * size_t(tps);
  }
  if (e == cudaSuccess) e = build_tiles(b, 128, 1);
  if (e == cudaSuccess) e = reset_state(b);
  if (e != cudaSuccess) { delete b; return RMRTLB_ECUDA; }
  *out = b;
  return RMRTLB_OK;
}

int rmrtlb_batch_destroy(rmrtlb_batch_t b) {
  if (!b) return RMRTLB_OK;
  drop_graph(b);
  delete b;
  return RMRTLB_OK;
}

int rmrtlb_batch_reset(rmrtlb_batch_t b) {
  if (!b) return RMRTLB_EINVAL;
  return reset_state(b) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

int rmrtlb_batch_step(rmrtlb_batch_t b, int n) {
  if (!b || n < 0) return RMRTLB_EINVAL;
  while (n > 0) {
    const bool at_boundary = b->step % b->check_every == 0 && b->cur == 0;
    if (at_boundary && n >= b->check_every) {
      if (chunk(b) != cudaSuccess) return RMRTLB_ECUDA;
      b->step += b->check_every;
      b->check_steps.push_back(b->step);
      n -= b->check_every;
      continue;
    }
    if (do_step(b) != cudaSuccess) return RMRTLB_ECUDA;
    b->cur ^= 1;
    ++b->step;
    --n;
    if (b->step % b->check_every == 0) {
      if (do_check(b) != cudaSuccess) return RMRTLB_ECUDA;
      b->check_steps.push_back(b->step);
    }
  }
  return RMRTLB_OK;
}

int rmrtlb_batch_run(rmrtlb_batch_t b, long long max_steps, long long* steps_done) {
  if (!b || max_steps < 0) return RMRTLB_EINVAL;
  const long long start = b->step;
  const long long per_poll = 8LL * b->check_every;
  std::vector<int> act;
  while (b->step - start < max_steps) {
    if (read_active(b, act)) return RMRTLB_ECUDA;
    size_t live = 0;
    for (size_t d = 0; d < act.size(); ++d)
      if (act[d] == 1) live += tiles_of(b->dom[d], b->width, b->rows);
    if (live == 0) break;
    // tile queue: once a quarter of the launched tiles belong to retired
    // domains, launch only the tiles of the domains still stepping
    if (4 * live < 3 * b->ntiles) {
      drop_graph(b);
      if (build_tiles(b, b->width, b->rows, &act) != cudaSuccess) return RMRTLB_ECUDA;
    }
    const long long left = max_steps - (b->step - start);
    const long long n = left < per_poll ? left : per_poll;
    const int rc = rmrtlb_batch_step(b, int(n));
    if (rc) return rc;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return RMRTLB_ECUDA;
  if (steps_done) *steps_done = b->step - start;
  return RMRTLB_OK;
}

int rmrtlb_batch_status(rmrtlb_batch_t b, double* residual, long long* steps_to_converge, int* active,
                        long long* steps_done) {
  if (!b) return RMRTLB_EINVAL;
  const size_t nd = b->dom.size();
  std::vector<double> st(2 * nd);
  std::vector<int> act(nd), conv(nd);
  if (cudaMemcpyAsync(st.data(), b->ws + b->L.status, st.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaMemcpyAsync(act.data(), b->ws + b->L.active, nd * sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(conv.data(), b->ws + b->L.conv, nd * sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  for (size_t d = 0; d < nd; ++d) {
    if (residual) residual[d] = b->check_steps.empty() ? -1.0 : st[2 * d];
    if (active) active[d] = act[d];
    if (steps_to_converge) {
      const int c = conv[d];   // 0-based index of the check at which the domain retired
      steps_to_converge[d] = (c >= 0 && size_t(c) < b->check_steps.size()) ? b->check_steps[c] : -1;
    }
  }
  if (steps_done) *steps_done = b->step;
  return RMRTLB_OK;
}

int rmrtlb_batch_tune(rmrtlb_batch_t b, int steps, int* width_out, int* rows_out, int* per_thread_out) {
  if (!b || steps < 1) return RMRTLB_EINVAL;
  float best = 1e30f;
  int best_w = b->width, best_r = b->rows, best_p = b->per_thread;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RMRTLB_ECUDA;
  // FP32: one node per thread, or the automatic mode (two while the batch fills the GPU)
  const int modes[2] = {1, 0};
  const int nmodes = b->storage == RMRTLB_ST_F32 ? 2 : 1;
  for (int mi = 0; mi < nmodes; ++mi)
    for (int r : kRows)
      for (int w : kWidths) {
        const int p = modes[mi];
        b->per_thread = p;
        if (build_tiles(b, w, r) != cudaSuccess) return RMRTLB_ECUDA;
        for (int i = 0; i < 2; ++i) { do_step(b); b->cur ^= 1; }
        cudaEventRecord(e0, b->stream);
        for (int i = 0; i < steps; ++i) { do_step(b); b->cur ^= 1; }
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return RMRTLB_ECUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_w = w; best_r = r; best_p = p; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graph(b);
  b->per_thread = best_p;
  if (build_tiles(b, best_w, best_r) != cudaSuccess || reset_state(b) != cudaSuccess) return RMRTLB_ECUDA;
  if (width_out) *width_out = best_w;
  if (rows_out) *rows_out = best_r;
  if (per_thread_out) *per_thread_out = best_p;
  return RMRTLB_OK;
}

int rmrtlb_batch_set_launch(rmrtlb_batch_t b, int tile_width, int tile_rows, int nodes_per_thread) {
  if (!b) return RMRTLB_EINVAL;
  bool w_ok = false, r_ok = false;
  for (int w : kWidths) w_ok = w_ok || w == tile_width;
  for (int r : kRows) r_ok = r_ok || r == tile_rows;
  const bool p_ok = nodes_per_thread == 1 ||
                    ((nodes_per_thread == 2 || nodes_per_thread == 0) && b->storage == RMRTLB_ST_F32);
  if (!w_ok || !r_ok || !p_ok) return RMRTLB_EINVAL;
  drop_graph(b);
  b->per_thread = nodes_per_thread;
  return build_tiles(b, tile_width, tile_rows) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

int rmrtlb_batch_set_populations(rmrtlb_batch_t b, int domain, const double* f) {
  if (!b || !f || domain < 0 || domain >= int(b->dom.size())) return RMRTLB_EINVAL;
  const size_t N = nodes_of(b->dom[domain]);
  int which = 0;
  if (domain_buffer(b, domain, &which)) return RMRTLB_ECUDA;
  const bool dev = dev_ptr(f);
  double* stage = at<double>(b, b->L.stage);
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int j = 0; j < b->q; ++j) {
    int e[3], jo = 0;
    lattice_dir(b->lat, j, e);
    for (int o = 0; o < b->q; ++o) {
      int eo[3];
      lattice_dir(b->lat, o, eo);
      if (eo[0] == -e[0] && eo[1] == -e[1] && eo[2] == -e[2]) jo = o;
    }
    // stage[0..N) = plane j (where the slot streams to), stage[N..2N) = plane jo (bounce)
    if (cudaMemcpyAsync(stage, f + size_t(j) * N, N * sizeof(double), k, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(stage + N, f + size_t(jo) * N, N * sizeof(double), k, b->stream) != cudaSuccess)
      return RMRTLB_ECUDA;
    if (dispatch(b, PlaneF{b, which, stage, j, 1, domain}) != cudaSuccess)
      return RMRTLB_ECUDA;
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

int rmrtlb_batch_get_populations(rmrtlb_batch_t b, int domain, double* f) {
  if (!b || !f || domain < 0 || domain >= int(b->dom.size())) return RMRTLB_EINVAL;
  const size_t N = nodes_of(b->dom[domain]);
  int which = 0;
  if (domain_buffer(b, domain, &which)) return RMRTLB_ECUDA;
  const bool dev = dev_ptr(f);
  double* stage = at<double>(b, b->L.stage);
  for (int j = 0; j < b->q; ++j) {
    double* plane = dev ? f + size_t(j) * N : stage;
    if (dispatch(b, PlaneF{b, which, plane, j, 0, domain}) != cudaSuccess)
      return RMRTLB_ECUDA;
    if (!dev && cudaMemcpyAsync(f + size_t(j) * N, stage, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream) !=
                    cudaSuccess)
      return RMRTLB_ECUDA;
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

int rmrtlb_batch_init_fields(rmrtlb_batch_t b, int domain, const double* rho, const double* u, int with_noneq) {
  if (!b || !rho || !u || domain < 0 || domain >= int(b->dom.size())) return RMRTLB_EINVAL;
  const size_t N = nodes_of(b->dom[domain]);
  int which = 0;
  if (domain_buffer(b, domain, &which)) return RMRTLB_ECUDA;
  double* stage = at<double>(b, b->L.stage);
  const double* r = rho;
  const double* v = u;
  if (!dev_ptr(rho)) {
    if (cudaMemcpyAsync(stage, rho, N * sizeof(double), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return RMRTLB_ECUDA;
    r = stage;
  }
  if (!dev_ptr(u)) {
    if (cudaMemcpyAsync(stage + N, u, size_t(b->d) * N * sizeof(double), cudaMemcpyHostToDevice, b->stream) !=
        cudaSuccess)
      return RMRTLB_ECUDA;
    v = stage + N;
  }
  if (dispatch(b, InitF{b, which, r, v, domain, with_noneq ? 1 : 0}) != cudaSuccess)
    return RMRTLB_ECUDA;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

int rmrtlb_batch_fields(rmrtlb_batch_t b, int domain, double* rho, double* u) {
  if (!b || domain < 0 || domain >= int(b->dom.size())) return RMRTLB_EINVAL;
  const size_t N = nodes_of(b->dom[domain]);
  int which = 0;
  if (domain_buffer(b, domain, &which)) return RMRTLB_ECUDA;
  double* stage = at<double>(b, b->L.stage);
  if (dispatch(b, FieldsF{b, which, domain, stage}) != cudaSuccess) return RMRTLB_ECUDA;
  const cudaMemcpyKind k1 = rho && dev_ptr(rho) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const cudaMemcpyKind k2 = u && dev_ptr(u) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (rho && cudaMemcpyAsync(rho, stage, N * sizeof(double), k1, b->stream) != cudaSuccess) return RMRTLB_ECUDA;
  if (u && cudaMemcpyAsync(u, stage + N, size_t(b->d) * N * sizeof(double), k2, b->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

}  // extern "C"
