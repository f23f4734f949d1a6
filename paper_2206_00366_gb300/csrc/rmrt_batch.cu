// Batched rD2Q9 lid-driven cavities: many independent rectangular domains
// (own size, spacing and viscosity) advanced together, one launch per step
// over a list of row tiles, with half-way bounce-back walls, a moving lid,
// a per-domain FP64 residual check and retirement of converged domains.
// Chunks of check_every steps plus their check are replayed as a CUDA graph.
//
// The paper has no boundaries and no batching; the collision of every node
// is the same Eq. (2-2-3) step as the single-domain kernels (shared code in
// rmrt_device.cuh).  Walls: a population whose source node x - e_j lies
// outside the domain is the node's own post-collision population in the
// opposite direction (half-way bounce-back); crossing the top wall (the lid,
// moving along x with U) adds 2 omega_j rho0 (c_j . U) / c_s^2, the linear
// term of the REDF (Eq. 3-3).
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/rmrtlb.h"
#include "rmrt_device.cuh"

namespace rmrt {

// Per-domain parameter block; the field names follow KParams so that the
// shared collision reads it.  Only what an unforced rD2Q9 NSE step needs.
template <typename CT>
struct BParams {
  int nx, ny;
  int kind;                 // KIND_NSE
  int pad_;
  unsigned long long off;   // element offset of the domain's population block
  unsigned long long uoff;  // element offset of its residual snapshot (2 planes)
  CT rho0, dt, source, cs2;
  CT mu2[3], s0, s1[3], s2h[3][3], soff[3], sfree;
  CT fh[3], advh[3], q19h[3];
  CT lid;                   // 2 omega_5 rho0 c_x U / c_s^2 (diagonal directions into the fluid)
  CT c[2];
  double wd[9];             // weights and rho0 in FP64 for population set/get
  double rho0d;
};

using L9 = Lat<LAT_D2Q9>;

__device__ __forceinline__ constexpr int opposite9(int j) {
  int r = 0;
  for (int k = 0; k < 9; ++k)
    if (L9::EX[k] == -L9::EX[j] && L9::EY[k] == -L9::EY[j]) r = k;
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

// Population j arriving at (x, y): pulled from (x - e_j) inside the domain,
// else bounced back from the node itself, with the lid term across the top.
template <typename CT, typename ST, int j>
__device__ __forceinline__ CT gather9(const ST* __restrict__ base, int x, int y, const BParams<CT>& sp) {
  constexpr int ex = L9::EX[j], ey = L9::EY[j], jo = opposite9(j);
  const int nx = sp.nx, ny = sp.ny;
  const int sx = x - ex, sy = y - ey;
  const bool inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
  const size_t N = size_t(nx) * ny;
  const size_t idx = inside ? size_t(j) * N + size_t(sy) * nx + sx : size_t(jo) * N + size_t(y) * nx + x;
  CT v = CT(__ldg(base + idx));
  if (ex != 0 && sy >= ny) v += CT(ex) * sp.lid;
  return v;
}

template <typename ST, typename CT>
__global__ void __launch_bounds__(256) batch_step_kernel(const ST* __restrict__ fin, ST* __restrict__ fout,
                                                         const BParams<CT>* __restrict__ dom,
                                                         const int4* __restrict__ tiles,
                                                         const int* __restrict__ active) {
  const int4 t = tiles[blockIdx.x];  // (domain, y, x0, width)
  if (!active[t.x]) return;          // retired: its last state stays in buffer A
  __shared__ BParams<CT> sp;
  load_params(sp, dom, t.x);
  const int x = t.z + int(threadIdx.x);
  if (int(threadIdx.x) >= t.w) return;
  const int y = t.y;
  const ST* base = fin + sp.off;
  Cube<LAT_D2Q9, CT> q;
  static_for<9>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L9::EX[j], ey = L9::EY[j];
    q.v[ex + 1][ey + 1][0] = gather9<CT, ST, j>(base, x, y, sp);
  });
  collide<LAT_D2Q9, false, false, true>(q, sp);
  const size_t N = size_t(sp.nx) * sp.ny;
  ST* out = fout + sp.off + size_t(y) * sp.nx + x;
  static_for<9>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L9::EX[j], ey = L9::EY[j];
    out[size_t(j) * N] = ST(q.v[ex + 1][ey + 1][0]);
  });
}

// Per-tile FP64 sums for the residual ||u - u_prev|| / ||u||: [0] sum
// |u - u_prev|^2, [1] sum |u|^2, [2] sum (rho - rho0).  Optionally writes
// the fields (rho_out, u_out: one domain, device, 3 planes).
template <typename ST, typename CT>
__global__ void __launch_bounds__(256) batch_check_kernel(const ST* __restrict__ fin,
                                                          const BParams<CT>* __restrict__ dom,
                                                          const int4* __restrict__ tiles,
                                                          const int* __restrict__ active,
                                                          double* __restrict__ uprev, int use_prev,
                                                          double* __restrict__ partials, int only_domain,
                                                          double* __restrict__ fields) {
  const int4 t = tiles[blockIdx.x];
  __shared__ double red[4][8];
  double acc[4] = {0, 0, 0, 0};
  const bool run = only_domain < 0 ? (active[t.x] != 0) : (t.x == only_domain);
  if (run) {
    __shared__ BParams<CT> sp;
    load_params(sp, dom, t.x);
    const int x = t.z + int(threadIdx.x);
    if (int(threadIdx.x) < t.w) {
      const int y = t.y;
      const ST* base = fin + sp.off;
      CT s0 = CT(0), sx = CT(0), sy = CT(0);
      static_for<9>([&](auto J) {
        constexpr int j = decltype(J)::value;
        constexpr int ex = L9::EX[j], ey = L9::EY[j];
        const CT v = gather9<CT, ST, j>(base, x, y, sp);
        s0 += v;
        if (ex) sx += CT(ex) * v;
        if (ey) sy += CT(ey) * v;
      });
      const CT rho = sp.rho0 + s0;
      const CT inv = CT(1) / rho;
      const double ux = double(sx * sp.c[0] * inv), uy = double(sy * sp.c[1] * inv);
      const size_t n = size_t(y) * sp.nx + x;
      const size_t N = size_t(sp.nx) * sp.ny;
      if (fields) {
        fields[n] = double(rho);
        fields[N + n] = ux;
        fields[2 * N + n] = uy;
      } else {
        double* up = uprev + sp.uoff;
        const double dx = ux - (use_prev ? up[n] : 0.0), dy = uy - (use_prev ? up[N + n] : 0.0);
        up[n] = ux;
        up[N + n] = uy;
        acc[0] = dx * dx + dy * dy;
        acc[1] = ux * ux + uy * uy;
        acc[2] = double(s0);
        acc[3] = isfinite(acc[1]) && isfinite(acc[2]) ? acc[1] : INFINITY;
      }
    }
  }
  if (fields) return;
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
// except the slots of the top row that stream into the lid: they bounce back
// as the direction jo with e_y = -1 and gain e_jo,x * lid, so they hold
// -e_jo,x * lid = e_j,x * lid.  grid (ceil(max nx / blockDim), ndomains).
template <typename ST, typename CT>
__global__ void batch_rest_kernel(ST* __restrict__ f, const BParams<CT>* __restrict__ dom) {
  const BParams<CT>& p = dom[blockIdx.y];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const size_t N = size_t(p.nx) * p.ny;
  const size_t n = size_t(p.ny - 1) * p.nx + x;
  static_for<9>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int ex = L9::EX[j], ey = L9::EY[j];
    if (ey == 1 && ex != 0) f[p.off + size_t(j) * N + n] = ST(CT(ex) * p.lid);
  });
}

// counters[0]: number of completed checks (a check with counters[0] > 0 has a
// previous snapshot).
__global__ void batch_bump_kernel(int* counters) {
  if (threadIdx.x == 0 && blockIdx.x == 0) counters[0] += 1;
}

// Canonical populations of one domain <-> storage (plane j).
// to_storage: A_j(y) = fbar_j(y + e_j) inside, else fbar_opp(y) - lid term;
// from_storage: fbar_j(x) = gather.
template <typename ST, typename CT>
__global__ void batch_plane_kernel(ST* __restrict__ f, double* __restrict__ plane, int j, int to_storage,
                                   const BParams<CT>* __restrict__ dom, int d) {
  __shared__ BParams<CT> sp;
  load_params(sp, dom, d);
  const int nx = sp.nx, ny = sp.ny;
  const size_t N = size_t(nx) * ny;
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = int(n % nx), y = int(n / nx);
  ST* base = f + sp.off;   // storage holds fbar - omega rho0 (omega_j = omega_opp(j))
  int ex = 0, ey = 0, jo = 0;
  static_for<9>([&](auto J) {
    constexpr int k = decltype(J)::value;
    constexpr int cx = L9::EX[k], cy = L9::EY[k], ko = opposite9(k);
    if (k == j) { ex = cx; ey = cy; jo = ko; }
  });
  if (to_storage) {
    // slot (x, y) of direction j holds the post-collision value that moves to (x + e_j)
    const int tx = x + ex, ty = y + ey;
    double v;
    if (tx >= 0 && tx < nx && ty >= 0 && ty < ny) {
      v = plane[N * 0 + size_t(ty) * nx + tx];
    } else {
      // it bounces back as direction jo at (x, y)
      v = plane[N * 1 + n];
      if (ty >= ny && ex != 0) v += double(ex) * double(sp.lid);   // undo the lid term of jo
    }
    base[size_t(j) * N + n] = ST(v - sp.wd[j] * sp.rho0d);
  } else {
    const int sx = x - ex, sy = y - ey;
    double v;
    if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) {
      v = double(base[size_t(j) * N + size_t(sy) * nx + sx]);
    } else {
      v = double(base[size_t(jo) * N + n]);
      if (sy >= ny && ex != 0) v += double(ex) * double(sp.lid);
    }
    plane[n] = v + sp.wd[j] * sp.rho0d;
  }
}

}  // namespace rmrt

using namespace rmrt;

namespace {

constexpr size_t kAlignB = 256;
size_t align_b(size_t v) { return (v + kAlignB - 1) / kAlignB * kAlignB; }
const int kWidths[4] = {32, 64, 128, 256};

struct BatchLayout {
  size_t fA, fB, uprev, dom, tiles, partials, tile_begin, active, status, conv, counters, cs2, stage, total;
  size_t pop_elems;          // elements of one population lattice (all domains)
  size_t max_tiles;
  size_t max_n;              // largest domain
};

size_t tiles_for(const std::vector<rmrtlb_domain>& d, int width) {
  size_t t = 0;
  for (const auto& x : d) t += size_t((x.nx + width - 1) / width) * x.ny;
  return t;
}

BatchLayout batch_layout(const std::vector<rmrtlb_domain>& d, int storage) {
  BatchLayout L;
  const size_t es = storage == RMRTLB_ST_F64 ? 8 : 4;
  size_t elems = 0, unodes = 0, maxn = 0;
  for (const auto& x : d) {
    const size_t n = size_t(x.nx) * x.ny;
    elems += align_b(9 * n * es) / es;
    unodes += 2 * n;
    maxn = n > maxn ? n : maxn;
  }
  L.pop_elems = elems;
  L.max_n = maxn;
  L.max_tiles = tiles_for(d, kWidths[0]);
  const size_t nd = d.size();
  const size_t psize = storage == RMRTLB_ST_F64 ? sizeof(BParams<double>) : sizeof(BParams<float>);
  L.fA = 0;
  L.fB = L.fA + align_b(elems * es);
  L.uprev = L.fB + align_b(elems * es);
  L.dom = L.uprev + align_b(unodes * sizeof(double));
  L.tiles = L.dom + align_b(nd * psize);
  L.partials = L.tiles + align_b(L.max_tiles * sizeof(int4));
  L.tile_begin = L.partials + align_b(L.max_tiles * 4 * sizeof(double));
  L.active = L.tile_begin + align_b((nd + 1) * sizeof(int));
  L.status = L.active + align_b(nd * sizeof(int));
  L.conv = L.status + align_b(2 * nd * sizeof(double));
  L.counters = L.conv + align_b(nd * sizeof(int));
  L.cs2 = L.counters + align_b(16 * sizeof(int));
  L.stage = L.cs2 + align_b(nd * sizeof(double));
  L.total = L.stage + align_b(2 * 9 * maxn * sizeof(double));
  return L;
}

bool rate_in(double s) { return s > 0.0 && s < 2.0 && isfinite(s); }

// Parameters of one cavity (the same derivation as rmrtlb_create: weights of
// Eq. 3-3-5, rates of Eq. 4-31, S_2 block of Eq. 5-8-1), in index units.
template <typename CT>
int domain_params(const rmrtlb_domain& D, double rho0, BParams<CT>& p) {
  memset(&p, 0, sizeof(p));
  if (D.nx < 1 || D.ny < 1 || !(D.dx > 0) || !(D.dy > 0) || !(D.nu > 0) || !(D.nu_bulk > 0)) return RMRTLB_EINVAL;
  const double c[2] = {D.dx, D.dy}, c2[2] = {D.dx * D.dx, D.dy * D.dy};
  const double cs2 = D.cs2 > 0 ? D.cs2 : fmin(c2[0], c2[1]) / 3.0;
  if (!(cs2 < c2[0] && cs2 < c2[1])) return RMRTLB_EINVAL;
  const double w5 = cs2 * cs2 / (4.0 * c2[0] * c2[1]);
  const double w1 = cs2 / (2.0 * c2[0]) - 2.0 * w5, w2 = cs2 / (2.0 * c2[1]) - 2.0 * w5;
  if (!(w5 > 0 && w1 > 0 && w2 > 0 && 1.0 - 2 * w1 - 2 * w2 - 4 * w5 > 0)) return RMRTLB_EINVAL;
  const double soff = 1.0 / (D.nu / cs2 + 0.5);
  double ss[2], sb[2];
  for (int a = 0; a < 2; ++a) {
    ss[a] = 1.0 / (2.0 * D.nu / (c2[a] - cs2) + 0.5);
    sb[a] = 1.0 / (2.0 * D.nu_bulk / (c2[a] - cs2) + 0.5);
    if (!rate_in(ss[a]) || !rate_in(sb[a])) return RMRTLB_EINVAL;
  }
  if (!rate_in(soff) || !rate_in(D.s_free)) return RMRTLB_EINVAL;
  double abar[2], b[2], den = 1.0;
  for (int a = 0; a < 2; ++a) {
    abar[a] = (1.0 / sb[a] - 1.0 / ss[a]) * (c2[a] - cs2) / 2.0;
    b[a] = 1.0 / (c2[a] - cs2);
    den += b[a] * ss[a] * abar[a];
  }
  p.nx = D.nx; p.ny = D.ny; p.kind = KIND_NSE;
  p.rho0 = CT(rho0); p.dt = CT(1); p.source = CT(0); p.cs2 = CT(cs2);
  for (int a = 0; a < 2; ++a) {
    p.mu2[a] = CT(cs2 / c2[a]);
    p.c[a] = CT(c[a]);
    for (int bb = 0; bb < 2; ++bb) {
      const double s2 = (a == bb ? ss[a] : 0.0) - ss[a] * abar[a] * b[bb] * ss[bb] / den;
      p.s2h[a][bb] = CT(s2 * c2[bb] / c2[a]);
    }
  }
  p.soff[0] = CT(soff); p.soff[1] = p.soff[2] = CT(D.s_free);
  p.sfree = CT(D.s_free); p.s0 = CT(D.s_free);
  for (int a = 0; a < 3; ++a) p.s1[a] = CT(D.s_free);
  p.lid = CT(2.0 * w5 * rho0 * c[0] * D.lid_u / cs2);
  const double w[9] = {1.0 - 2 * w1 - 2 * w2 - 4 * w5, w1, w2, w1, w2, w5, w5, w5, w5};
  for (int j = 0; j < 9; ++j) p.wd[j] = w[j];
  p.rho0d = rho0;
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
  std::vector<rmrtlb_domain> dom;
  std::vector<size_t> off;          // element offsets per domain
  std::vector<int> tile_begin_host;
  BatchLayout L;
  int storage;
  char* ws;
  cudaStream_t stream;
  int width;                        // tile width (threads per block)
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

cudaError_t build_tiles(rmrtlb_batch* b, int width) {
  std::vector<int4> t;
  std::vector<int> tb(b->dom.size() + 1, 0);
  for (size_t d = 0; d < b->dom.size(); ++d) {
    tb[d] = int(t.size());
    const auto& D = b->dom[d];
    for (int y = 0; y < D.ny; ++y)
      for (int x0 = 0; x0 < D.nx; x0 += width) t.push_back(make_int4(int(d), y, x0, D.nx - x0 < width ? D.nx - x0 : width));
  }
  tb[b->dom.size()] = int(t.size());
  b->ntiles = t.size();
  b->width = width;
  b->tile_begin_host = tb;
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

template <typename ST, typename CT>
cudaError_t launch_step(rmrtlb_batch* b) {
  const ST* fin = at<ST>(b, b->cur == 0 ? b->L.fA : b->L.fB);
  ST* fout = at<ST>(b, b->cur == 0 ? b->L.fB : b->L.fA);
  batch_step_kernel<ST, CT><<<unsigned(b->ntiles), b->width, 0, b->stream>>>(
      fin, fout, at<BParams<CT>>(b, b->L.dom), at<int4>(b, b->L.tiles), at<int>(b, b->L.active));
  return cudaGetLastError();
}

template <typename ST, typename CT>
cudaError_t launch_check(rmrtlb_batch* b, double* fields, int only_domain) {
  const ST* fin = at<ST>(b, b->cur == 0 ? b->L.fA : b->L.fB);
  batch_check_kernel<ST, CT><<<unsigned(b->ntiles), b->width, 0, b->stream>>>(
      fin, at<BParams<CT>>(b, b->L.dom), at<int4>(b, b->L.tiles), at<int>(b, b->L.active),
      at<double>(b, b->L.uprev), 1, at<double>(b, b->L.partials), only_domain, fields);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || fields) return e;
  batch_reduce_kernel<<<unsigned(b->dom.size()), 256, 0, b->stream>>>(
      at<double>(b, b->L.partials), at<int>(b, b->L.tile_begin), at<int>(b, b->L.active),
      at<double>(b, b->L.status), at<int>(b, b->L.conv), at<int>(b, b->L.counters), at<double>(b, b->L.cs2), b->tol);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_bump_kernel<<<1, 32, 0, b->stream>>>(at<int>(b, b->L.counters));
  return cudaGetLastError();
}

cudaError_t do_step(rmrtlb_batch* b) {
  return b->storage == RMRTLB_ST_F64 ? launch_step<double, double>(b) : launch_step<float, float>(b);
}
cudaError_t do_check(rmrtlb_batch* b, double* fields = nullptr, int only = -1) {
  return b->storage == RMRTLB_ST_F64 ? launch_check<double, double>(b, fields, only)
                                     : launch_check<float, float>(b, fields, only);
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
  cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
  if (e != cudaSuccess) return e;
  return cudaSuccess;   // chunk_direct's parity changes cancel: check_every is even
}

cudaError_t reset_state(rmrtlb_batch* b) {
  const size_t es = b->storage == RMRTLB_ST_F64 ? 8 : 4;
  cudaError_t e = cudaMemsetAsync(b->ws + b->L.fA, 0, b->L.pop_elems * es, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.fB, 0, b->L.pop_elems * es, b->stream);
  if (e == cudaSuccess) {
    int maxnx = 1;
    for (const auto& d : b->dom) maxnx = d.nx > maxnx ? d.nx : maxnx;
    const dim3 grid(unsigned((maxnx + 127) / 128), unsigned(b->dom.size()));
    if (b->storage == RMRTLB_ST_F64)
      batch_rest_kernel<double, double><<<grid, 128, 0, b->stream>>>(at<double>(b, b->L.fA),
                                                                   at<BParams<double>>(b, b->L.dom));
    else
      batch_rest_kernel<float, float><<<grid, 128, 0, b->stream>>>(at<float>(b, b->L.fA),
                                                                 at<BParams<float>>(b, b->L.dom));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.uprev, 0, b->L.dom - b->L.uprev, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws + b->L.counters, 0, 16 * sizeof(int), b->stream);
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

}  // namespace

extern "C" {

int rmrtlb_batch_workspace_bytes(int ndomains, const rmrtlb_domain* domains, int storage, size_t* bytes) {
  if (ndomains < 1 || !domains || !bytes || (storage != RMRTLB_ST_F32 && storage != RMRTLB_ST_F64))
    return RMRTLB_EINVAL;
  std::vector<rmrtlb_domain> d(domains, domains + ndomains);
  for (const auto& x : d)
    if (x.nx < 1 || x.ny < 1 || x.ny > (1 << 30) / 9 || double(x.nx) * x.ny > 2.0e8) return RMRTLB_EINVAL;
  *bytes = batch_layout(d, storage).total;
  return RMRTLB_OK;
}

int rmrtlb_batch_create(rmrtlb_batch_t* out, int ndomains, const rmrtlb_domain* domains, int storage, double rho0,
                        int check_every, double tol, void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return RMRTLB_EINVAL;
  *out = nullptr;
  size_t need = 0;
  int rc = rmrtlb_batch_workspace_bytes(ndomains, domains, storage, &need);
  if (rc) return rc;
  if (!workspace || reinterpret_cast<size_t>(workspace) % kAlignB) return RMRTLB_EINVAL;
  if (workspace_bytes < need) return RMRTLB_ENOMEM;
  if (check_every < 2 || !(tol > 0) || !isfinite(rho0)) return RMRTLB_EINVAL;
  rmrtlb_batch* b = new (std::nothrow) rmrtlb_batch();
  if (!b) return RMRTLB_ENOMEM;
  b->dom.assign(domains, domains + ndomains);
  b->storage = storage;
  b->L = batch_layout(b->dom, storage);
  b->ws = static_cast<char*>(workspace);
  b->stream = static_cast<cudaStream_t>(stream);
  b->check_every = check_every + (check_every & 1);
  b->tol = tol;
  b->graph_ok = false;
  // parameter blocks and population offsets
  const size_t es = storage == RMRTLB_ST_F64 ? 8 : 4;
  size_t off = 0, uoff = 0;
  std::vector<char> params(ndomains * (storage == RMRTLB_ST_F64 ? sizeof(BParams<double>) : sizeof(BParams<float>)));
  for (int d = 0; d < ndomains; ++d) {
    const size_t n = size_t(b->dom[d].nx) * b->dom[d].ny;
    b->off.push_back(off);
    if (storage == RMRTLB_ST_F64) {
      BParams<double> p;
      rc = domain_params(b->dom[d], rho0, p);
      p.off = off; p.uoff = uoff;
      memcpy(params.data() + d * sizeof(p), &p, sizeof(p));
    } else {
      BParams<float> p;
      rc = domain_params(b->dom[d], rho0, p);
      p.off = off; p.uoff = uoff;
      memcpy(params.data() + d * sizeof(p), &p, sizeof(p));
    }
    if (rc) { delete b; return rc; }
    off += align_b(9 * n * es) / es;
    uoff += 2 * n;
  }
  std::vector<double> cs2(ndomains);
  for (int d = 0; d < ndomains; ++d) {
    const double m = fmin(b->dom[d].dx, b->dom[d].dy);
    cs2[d] = b->dom[d].cs2 > 0 ? b->dom[d].cs2 : m * m / 3.0;
  }
  cudaError_t e = cudaMemcpyAsync(b->ws + b->L.dom, params.data(), params.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + b->L.cs2, cs2.data(), cs2.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = build_tiles(b, 128);
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

int rmrtlb_batch_tune(rmrtlb_batch_t b, int steps, int* width_out) {
  if (!b || steps < 1) return RMRTLB_EINVAL;
  float best = 1e30f;
  int best_w = b->width;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RMRTLB_ECUDA;
  for (int w : kWidths) {
    if (build_tiles(b, w) != cudaSuccess) return RMRTLB_ECUDA;
    for (int i = 0; i < 2; ++i) { do_step(b); b->cur ^= 1; }
    cudaEventRecord(e0, b->stream);
    for (int i = 0; i < steps; ++i) { do_step(b); b->cur ^= 1; }
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return RMRTLB_ECUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_w = w; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graph(b);
  if (build_tiles(b, best_w) != cudaSuccess || reset_state(b) != cudaSuccess) return RMRTLB_ECUDA;
  if (width_out) *width_out = best_w;
  return RMRTLB_OK;
}

int rmrtlb_batch_set_populations(rmrtlb_batch_t b, int domain, const double* f) {
  if (!b || !f || domain < 0 || domain >= int(b->dom.size())) return RMRTLB_EINVAL;
  const size_t N = size_t(b->dom[domain].nx) * b->dom[domain].ny;
  const bool dev = dev_ptr(f);
  double* stage = at<double>(b, b->L.stage);
  for (int j = 0; j < 9; ++j) {
    static const int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    // stage[0..N) = plane j (where the slot streams to), stage[N..2N) = plane opp(j) (bounce)
    const double* pj = f + size_t(j) * N;
    const double* po = f + size_t(opp[j]) * N;
    cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(stage, pj, N * sizeof(double), k, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(stage + N, po, N * sizeof(double), k, b->stream) != cudaSuccess)
      return RMRTLB_ECUDA;
    const unsigned grid = unsigned((N + 255) / 256);
    if (b->storage == RMRTLB_ST_F64)
      batch_plane_kernel<double, double><<<grid, 256, 0, b->stream>>>(at<double>(b, b->cur == 0 ? b->L.fA : b->L.fB),
                                                                      stage, j, 1, at<BParams<double>>(b, b->L.dom),
                                                                      domain);
    else
      batch_plane_kernel<float, float><<<grid, 256, 0, b->stream>>>(at<float>(b, b->cur == 0 ? b->L.fA : b->L.fB),
                                                                    stage, j, 1, at<BParams<float>>(b, b->L.dom),
                                                                    domain);
    if (cudaGetLastError() != cudaSuccess) return RMRTLB_ECUDA;
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

// Current buffer of a domain: a retired domain's state stays in A.
static int domain_buffer(rmrtlb_batch* b, int domain, int* which) {
  int act = 1;
  if (cudaMemcpyAsync(&act, b->ws + b->L.active + domain * sizeof(int), sizeof(int), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  *which = act == 1 ? b->cur : 0;
  return RMRTLB_OK;
}

int rmrtlb_batch_get_populations(rmrtlb_batch_t b, int domain, double* f) {
  if (!b || !f || domain < 0 || domain >= int(b->dom.size())) return RMRTLB_EINVAL;
  const size_t N = size_t(b->dom[domain].nx) * b->dom[domain].ny;
  int which = 0;
  if (domain_buffer(b, domain, &which)) return RMRTLB_ECUDA;
  const bool dev = dev_ptr(f);
  double* stage = at<double>(b, b->L.stage);
  for (int j = 0; j < 9; ++j) {
    double* plane = dev ? f + size_t(j) * N : stage;
    const unsigned grid = unsigned((N + 255) / 256);
    if (b->storage == RMRTLB_ST_F64)
      batch_plane_kernel<double, double><<<grid, 256, 0, b->stream>>>(at<double>(b, which == 0 ? b->L.fA : b->L.fB),
                                                                      plane, j, 0, at<BParams<double>>(b, b->L.dom),
                                                                      domain);
    else
      batch_plane_kernel<float, float><<<grid, 256, 0, b->stream>>>(at<float>(b, which == 0 ? b->L.fA : b->L.fB),
                                                                    plane, j, 0, at<BParams<float>>(b, b->L.dom),
                                                                    domain);
    if (cudaGetLastError() != cudaSuccess) return RMRTLB_ECUDA;
    if (!dev && cudaMemcpyAsync(f + size_t(j) * N, stage, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream) !=
                    cudaSuccess)
      return RMRTLB_ECUDA;
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

int rmrtlb_batch_fields(rmrtlb_batch_t b, int domain, double* rho, double* u) {
  if (!b || domain < 0 || domain >= int(b->dom.size())) return RMRTLB_EINVAL;
  const size_t N = size_t(b->dom[domain].nx) * b->dom[domain].ny;
  int which = 0;
  if (domain_buffer(b, domain, &which)) return RMRTLB_ECUDA;
  double* stage = at<double>(b, b->L.stage);
  const int cur = b->cur;
  b->cur = which;
  const cudaError_t e = do_check(b, stage, domain);
  b->cur = cur;
  if (e != cudaSuccess) return RMRTLB_ECUDA;
  const cudaMemcpyKind k1 = rho && dev_ptr(rho) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const cudaMemcpyKind k2 = u && dev_ptr(u) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (rho && cudaMemcpyAsync(rho, stage, N * sizeof(double), k1, b->stream) != cudaSuccess) return RMRTLB_ECUDA;
  if (u && cudaMemcpyAsync(u, stage + N, 2 * N * sizeof(double), k2, b->stream) != cudaSuccess) return RMRTLB_ECUDA;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

}  // extern "C"
