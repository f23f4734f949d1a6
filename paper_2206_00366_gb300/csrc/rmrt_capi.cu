// Host side of the C ABI declared in include/rmrtlb.h: parameter derivation
// (Sec. III weights, Eq. 4-31 rates, Eq. 5-8-1 S_2 block), workspace layout,
// host/device transfers and the launch sequence of one solver.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "../../include/rmrtlb.h"
#include "rmrt_aux.cuh"
#include "rmrt_device.cuh"
#include "rmrt_params.h"

namespace rmrt {

// Fixed-order FP64 sum of nblk rows of 8 partial sums (7 used).
__global__ void __launch_bounds__(256) finalize_kernel(const double* __restrict__ partials, size_t nblk,
                                                       double* __restrict__ out) {
  __shared__ double sm[7][256];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (size_t i = threadIdx.x; i < nblk; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < 7; ++k) acc[k] += partials[i * 8 + k];
#pragma unroll
  for (int k = 0; k < 7; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 7; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 7) out[threadIdx.x] = sm[threadIdx.x][0];
  if (threadIdx.x == 7) out[7] = 0.0;
}

cudaError_t launch_finalize(const double* partials, size_t nblk, double* out, cudaStream_t s) {
  finalize_kernel<<<1, 256, 0, s>>>(partials, nblk, out);
  return cudaGetLastError();
}

}  // namespace rmrt

using namespace rmrt;

namespace {

constexpr int kSlots = 2;          // 0: periodic check in rmrtlb_step, 1: rmrtlb_stats
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int lattice_q(int lat) { return lat == RMRTLB_D2Q9 ? 9 : (lat == RMRTLB_D3Q19 ? 19 : 27); }
int lattice_d(int lat) { return lat == RMRTLB_D2Q9 ? 2 : 3; }
size_t storage_size(int st) { return st == RMRTLB_ST_F64 ? 8 : (st == RMRTLB_ST_F32 ? 4 : 2); }

void lattice_dir(int lat, int j, int e[3]) {
  if (lat == RMRTLB_D2Q9) {
    e[0] = Lat<LAT_D2Q9>::EX[j]; e[1] = Lat<LAT_D2Q9>::EY[j]; e[2] = 0;
  } else {
    e[0] = Dirs27::EX[j]; e[1] = Dirs27::EY[j]; e[2] = Dirs27::EZ[j];
  }
}

int block_x(int nx) {
  if (nx >= 128) return 128;
  return ((nx + 31) / 32) * 32;
}

// Blocks of the grid-stride check kernel (one partial row each).
size_t check_blocks(size_t N) {
  const size_t b = (N + CHECK_THREADS - 1) / CHECK_THREADS;
  return b < size_t(CHECK_MAX_BLOCKS) ? b : size_t(CHECK_MAX_BLOCKS);
}

struct Layout {
  size_t fA, fB, stage, uprev, partials, stats, flags, total, nblk;
};

Layout make_layout(int lat, int nx, int ny, int nz, int st) {
  const size_t N = size_t(nx) * ny * nz;
  const int q = lattice_q(lat), d = lattice_d(lat);
  Layout L;
  L.nblk = check_blocks(N);
  const size_t pop = align_up(q * N * storage_size(st));
  L.fA = 0;
  L.fB = L.fA + pop;
  L.stage = L.fB + pop;
  L.uprev = L.stage + align_up((d + 1) * N * sizeof(double));
  L.partials = L.uprev + align_up(d * N * sizeof(double));
  L.stats = L.partials + align_up(L.nblk * 8 * sizeof(double));
  L.flags = L.stats + align_up(kSlots * 8 * sizeof(double));
  L.total = L.flags + align_up(kSlots * sizeof(int));
  return L;
}

bool valid_dims(int lat, int nx, int ny, int nz) {
  if (lat < 0 || lat > 2 || nx < 1 || ny < 1 || nz < 1) return false;
  if (lat == RMRTLB_D2Q9 && nz != 1) return false;
  if (ny > 65535 || nz > 65535) return false;             // grid.y, grid.z limits
  const double N = double(nx) * ny * nz;
  return N * lattice_q(lat) < 9.0e18 && N < 2147483647.0;
}

// All constants of a solver, in FP64.
struct Consts {
  int lat, d, q, kind, forced, storage, central;
  int nx, ny, nz;
  size_t N;
  double c[3], cs2, dt, rho0, source;
  double w[27];
  double s0, s1[3], s2[3][3], soff[3], sfree;
  double force[3], adv[3];
};

bool rate_ok(double s) { return s > 0.0 && s < 2.0 && isfinite(s); }

// Weights from the velocity-moment constraints (Sec. III): rD2Q9 Eq. (3-3-5),
// rD3Q27 Eq. (3-3-8) with omega_19 = c_s^6/(8 c1^2 c2^2 c3^2), rD3Q19 with
// omega_19 = 0; omega_0 = 1 - sum of the others.
int derive_weights(Consts& k) {
  const double cs2 = k.cs2;
  double c2[3] = {k.c[0] * k.c[0], k.c[1] * k.c[1], k.c[2] * k.c[2]};
  double wax[3] = {0, 0, 0}, wedge[3] = {0, 0, 0}, wcorner = 0;  // edge: xy, xz, yz
  if (k.lat == RMRTLB_D2Q9) {
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
int derive_rates(Consts& k, const rmrtlb_params& p) {
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
KParams<CT> to_kparams(const Consts& k) {
  KParams<CT> p;
  memset(&p, 0, sizeof(p));
  p.nx = k.nx; p.ny = k.ny; p.nz = k.nz;
  p.kind = k.kind; p.forced = k.forced; p.N = k.N;
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
  const bool scaled = k.storage == RMRTLB_ST_F16 || k.storage == RMRTLB_ST_BF16;
  for (int j = 0; j < 27; ++j) {
    if (j < k.q) {
      // 16-bit storage: power of two nearest 1/omega_j (exact to apply and
      // undo); 32/64-bit storage is unscaled
      const int e = scaled ? int(lround(-log2(k.w[j]))) : 0;
      p.sc[j] = CT(ldexp(1.0, e));
      p.sinv[j] = CT(ldexp(1.0, -e));
      p.wd[j] = k.w[j];
    }
  }
  p.s0 = CT(k.s0); p.sfree = CT(k.sfree);
  return p;
}

}  // namespace

struct rmrtlb_solver {
  Consts k;
  Layout L;
  char* ws;
  cudaStream_t stream;
  KParams<double> kp64;
  KParams<float> kp32;
  int cur;            // 0: populations in fA, 1: in fB
  long long step;
  int check_every;
  int pairs;          // step kernel handles two nodes per thread (nx even)
  bool has_prev;      // a periodic check wrote the residual snapshot
  long long slot_step[kSlots];
  bool slot_prev[kSlots];
  bool slot_valid[kSlots];
};

namespace {

void* pop_ptr(rmrtlb_solver* s, int which) { return s->ws + (which == 0 ? s->L.fA : s->L.fB); }
double* stage_ptr(rmrtlb_solver* s) { return reinterpret_cast<double*>(s->ws + s->L.stage); }

LaunchArgs base_args(rmrtlb_solver* s, Op op) {
  LaunchArgs a;
  memset(&a, 0, sizeof(a));
  a.op = op;
  a.storage = s->k.storage;
  a.central = s->k.central;
  a.kp64 = &s->kp64;
  a.kp32 = &s->kp32;
  const int bx = block_x(s->k.nx);
  a.block = dim3(bx, 1, 1);
  a.grid = dim3((s->k.nx + bx - 1) / bx, s->k.ny, s->k.nz);
  a.stream = s->stream;
  return a;
}

cudaError_t launch(rmrtlb_solver* s, const LaunchArgs& a) {
  using Fn = cudaError_t (*)(const LaunchArgs&);
  static const Fn table[3][4] = {
      {launch_d2q9_f64, launch_d2q9_f32, launch_d2q9_f16, launch_d2q9_bf16},
      {launch_d3q19_f64, launch_d3q19_f32, launch_d3q19_f16, launch_d3q19_bf16},
      {launch_d3q27_f64, launch_d3q27_f32, launch_d3q27_f16, launch_d3q27_bf16}};
  return table[s->k.lat][s->k.storage](a);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Run the check kernel into a stats slot (and optionally the field outputs).
cudaError_t run_check(rmrtlb_solver* s, int slot, double* rho_out, double* u_out, bool with_sums,
                      bool write_prev) {
  cudaError_t e;
  int* flags = reinterpret_cast<int*>(s->ws + s->L.flags) + slot;
  double* partials = reinterpret_cast<double*>(s->ws + s->L.partials);
  double* stats = reinterpret_cast<double*>(s->ws + s->L.stats) + 8 * slot;
  if (with_sums) {
    e = cudaMemsetAsync(flags, 0, sizeof(int), s->stream);
    if (e != cudaSuccess) return e;
  }
  LaunchArgs a = base_args(s, OP_CHECK);
  a.grid = dim3(unsigned(s->L.nblk), 1, 1);
  a.block = dim3(CHECK_THREADS, 1, 1);
  a.fin = pop_ptr(s, s->cur);
  a.rho_out = rho_out;
  a.u_out = u_out;
  if (with_sums) {
    a.uprev = reinterpret_cast<double*>(s->ws + s->L.uprev);
    a.use_prev = s->has_prev ? 1 : 0;
    a.write_prev = write_prev ? 1 : 0;
    a.partials = partials;
    a.flags = flags;
  }
  e = launch(s, a);
  if (e != cudaSuccess) return e;
  if (with_sums) {
    e = launch_finalize(partials, s->L.nblk, stats, s->stream);
    if (e != cudaSuccess) return e;
    s->slot_step[slot] = s->step;
    s->slot_prev[slot] = s->has_prev;
    s->slot_valid[slot] = true;
    if (write_prev) s->has_prev = true;
  }
  return cudaSuccess;
}

int read_slot(rmrtlb_solver* s, int slot, double out[8]) {
  double raw[8];
  int flags = 0;
  if (cudaMemcpyAsync(raw, s->ws + s->L.stats + slot * 8 * sizeof(double), sizeof(raw), cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess ||
      cudaMemcpyAsync(&flags, s->ws + s->L.flags + slot * sizeof(int), sizeof(int), cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  out[0] = double(s->k.N) * s->k.rho0 + raw[0];
  out[1] = raw[1]; out[2] = raw[2]; out[3] = raw[3];
  out[4] = raw[4];
  out[5] = s->slot_prev[slot] && raw[6] > 0 ? sqrt(raw[5] / raw[6]) : -1.0;
  out[6] = double(s->slot_step[slot]);
  out[7] = double(flags);
  return flags ? RMRTLB_EUNSTABLE : RMRTLB_OK;
}

}  // namespace

extern "C" {

const char* rmrtlb_strerror(int status) {
  switch (status) {
    case RMRTLB_OK: return "ok";
    case RMRTLB_EINVAL: return "invalid argument";
    case RMRTLB_ENOMEM: return "workspace too small";
    case RMRTLB_ECUDA: return "CUDA runtime error";
    case RMRTLB_EUNSTABLE: return "unstable state (NaN/Inf, density <= 0 or |u| >= c_s)";
    case RMRTLB_ETOOBIG: return "input larger than the fixed internal buffer allows";
    default: return "unknown status";
  }
}

int rmrtlb_lattice_info(int lattice, int* q, int* d, int* e) {
  if (lattice < 0 || lattice > 2) return RMRTLB_EINVAL;
  if (q) *q = lattice_q(lattice);
  if (d) *d = lattice_d(lattice);
  if (e)
    for (int j = 0; j < lattice_q(lattice); ++j) lattice_dir(lattice, j, e + 3 * j);
  return RMRTLB_OK;
}

int rmrtlb_workspace_bytes(int lattice, int nx, int ny, int nz, int storage, size_t* bytes) {
  if (!bytes || !valid_dims(lattice, nx, ny, nz) || storage < 0 || storage > 3) return RMRTLB_EINVAL;
  *bytes = make_layout(lattice, nx, ny, nz, storage).total;
  return RMRTLB_OK;
}

int rmrtlb_create(rmrtlb_t* solver, int lattice, int nx, int ny, int nz, double dx, double dy, double dz,
                  double dt, const rmrtlb_params* params, int eq_kind, int basis, int storage, void* workspace,
                  size_t workspace_bytes, void* stream) {
  if (!solver || !params || !valid_dims(lattice, nx, ny, nz)) return RMRTLB_EINVAL;
  *solver = nullptr;
  if (eq_kind < 0 || eq_kind > 3 || basis < 0 || basis > 1 || storage < 0 || storage > 3) return RMRTLB_EINVAL;
  if (!(dt > 0) || !(dx > 0) || !(dy > 0) || (lattice != RMRTLB_D2Q9 && !(dz > 0))) return RMRTLB_EINVAL;
  if (!workspace || (reinterpret_cast<size_t>(workspace) % kAlign) != 0) return RMRTLB_EINVAL;
  const Layout L = make_layout(lattice, nx, ny, nz, storage);
  if (workspace_bytes < L.total) return RMRTLB_ENOMEM;

  Consts k;
  memset(&k, 0, sizeof(k));
  k.lat = lattice; k.d = lattice_d(lattice); k.q = lattice_q(lattice);
  k.kind = eq_kind; k.storage = storage; k.central = basis;
  k.nx = nx; k.ny = ny; k.nz = nz; k.N = size_t(nx) * ny * nz;
  k.dt = dt;
  const double sp[3] = {dx, dy, lattice == RMRTLB_D2Q9 ? 1.0 : dz};
  double cmin2 = 1e300;
  for (int a = 0; a < 3; ++a) {
    k.c[a] = sp[a] / dt;
    if (a < k.d) cmin2 = fmin(cmin2, k.c[a] * k.c[a]);
  }
  k.cs2 = params->cs2 > 0 ? params->cs2 : cmin2 / 3.0;
  if (!(k.cs2 < cmin2)) return RMRTLB_EINVAL;
  k.rho0 = params->rho0;
  if (!isfinite(k.rho0)) return RMRTLB_EINVAL;
  k.source = params->source;
  for (int a = 0; a < 3; ++a) {
    k.force[a] = a < k.d ? params->force[a] : 0.0;
    k.adv[a] = a < k.d ? params->adv[a] : 0.0;
  }
  const bool nse = eq_kind == RMRTLB_EQ_NSE || eq_kind == RMRTLB_EQ_NSE_HELUO;
  k.forced = (k.source != 0.0) || (nse && (k.force[0] != 0.0 || k.force[1] != 0.0 || k.force[2] != 0.0));
  if (!nse) for (int a = 0; a < 3; ++a) k.force[a] = 0.0;
  int rc = derive_weights(k);
  if (rc) return rc;
  rc = derive_rates(k, *params);
  if (rc) return rc;
  if (params->check_every < 0) return RMRTLB_EINVAL;

  rmrtlb_solver* s = new (std::nothrow) rmrtlb_solver;
  if (!s) return RMRTLB_ENOMEM;
  memset(s, 0, sizeof(*s));
  s->k = k;
  s->L = L;
  s->ws = static_cast<char*>(workspace);
  s->stream = static_cast<cudaStream_t>(stream);
  s->kp64 = to_kparams<double>(k);
  s->kp32 = to_kparams<float>(k);
  s->check_every = params->check_every;
  s->pairs = (nx % 2 == 0);
  *solver = s;
  return RMRTLB_OK;
}

int rmrtlb_destroy(rmrtlb_t solver) {
  delete solver;
  return RMRTLB_OK;
}

int rmrtlb_get_constants(rmrtlb_t s, double* out, int n) {
  if (!s || !out || n < 48) return RMRTLB_EINVAL;
  for (int i = 0; i < 48; ++i) out[i] = 0.0;
  out[0] = s->k.cs2;
  for (int a = 0; a < 3; ++a) out[1 + a] = s->k.c[a];
  for (int j = 0; j < s->k.q; ++j) out[4 + j] = s->k.w[j];
  out[31] = s->k.s0;
  for (int a = 0; a < 3; ++a) out[32 + a] = s->k.s1[a];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) out[35 + 3 * i + j] = s->k.s2[i][j];
  for (int i = 0; i < 3; ++i) out[44 + i] = s->k.soff[i];
  out[47] = s->k.sfree;
  return RMRTLB_OK;
}

int rmrtlb_init_equilibrium(rmrtlb_t s, const double* rho, const double* u) {
  if (!s || !rho) return RMRTLB_EINVAL;
  const bool nse = s->k.kind == RMRTLB_EQ_NSE || s->k.kind == RMRTLB_EQ_NSE_HELUO;
  if (nse && !u) return RMRTLB_EINVAL;
  const size_t N = s->k.N;
  const double* drho = rho;
  const double* du = u;
  bool synced = false;
  if (!is_device_ptr(rho)) {
    if (cudaMemcpyAsync(stage_ptr(s), rho, N * sizeof(double), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
      return RMRTLB_ECUDA;
    drho = stage_ptr(s);
    synced = true;
  }
  if (nse && !is_device_ptr(u)) {
    if (cudaMemcpyAsync(stage_ptr(s) + N, u, s->k.d * N * sizeof(double), cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
      return RMRTLB_ECUDA;
    du = stage_ptr(s) + N;
    synced = true;
  }
  LaunchArgs a = base_args(s, OP_INIT_EQ);
  s->cur = 0;
  a.fout = pop_ptr(s, 0);
  a.rho = drho;
  a.u = nse ? du : drho;
  if (launch(s, a) != cudaSuccess) return RMRTLB_ECUDA;
  s->step = 0;
  s->has_prev = false;
  if (synced && cudaStreamSynchronize(s->stream) != cudaSuccess) return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

int rmrtlb_set_populations(rmrtlb_t s, const double* f) {
  if (!s || !f) return RMRTLB_EINVAL;
  const size_t N = s->k.N;
  const bool dev = is_device_ptr(f);
  for (int j = 0; j < s->k.q; ++j) {
    double* plane = const_cast<double*>(f) + size_t(j) * N;
    if (!dev) {
      if (cudaMemcpyAsync(stage_ptr(s), plane, N * sizeof(double), cudaMemcpyHostToDevice, s->stream) !=
          cudaSuccess)
        return RMRTLB_ECUDA;
      plane = stage_ptr(s);
    }
    LaunchArgs a = base_args(s, OP_PLANE);
    a.fout = pop_ptr(s, s->cur);
    a.plane = plane;
    a.j = j;
    a.to_storage = 1;
    if (launch(s, a) != cudaSuccess) return RMRTLB_ECUDA;
  }
  s->step = 0;
  s->has_prev = false;
  if (!dev && cudaStreamSynchronize(s->stream) != cudaSuccess) return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

int rmrtlb_get_populations(rmrtlb_t s, double* f) {
  if (!s || !f) return RMRTLB_EINVAL;
  const size_t N = s->k.N;
  const bool dev = is_device_ptr(f);
  for (int j = 0; j < s->k.q; ++j) {
    double* plane = dev ? f + size_t(j) * N : stage_ptr(s);
    LaunchArgs a = base_args(s, OP_PLANE);
    a.fout = pop_ptr(s, s->cur);
    a.plane = plane;
    a.j = j;
    a.to_storage = 0;
    if (launch(s, a) != cudaSuccess) return RMRTLB_ECUDA;
    if (!dev && cudaMemcpyAsync(f + size_t(j) * N, plane, N * sizeof(double), cudaMemcpyDeviceToHost,
                                s->stream) != cudaSuccess)
      return RMRTLB_ECUDA;
  }
  if (!dev && cudaStreamSynchronize(s->stream) != cudaSuccess) return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

int rmrtlb_step(rmrtlb_t s, int n) {
  if (!s || n < 0) return RMRTLB_EINVAL;
  for (int i = 0; i < n; ++i) {
    LaunchArgs a = base_args(s, OP_STEP);
    if (s->pairs) {
      const int half = s->k.nx / 2;
      const int bx = block_x(half);
      a.pairs = 1;
      a.block = dim3(bx, 1, 1);
      a.grid = dim3((half + bx - 1) / bx, s->k.ny, s->k.nz);
    }
    a.fin = pop_ptr(s, s->cur);
    a.fout = pop_ptr(s, 1 - s->cur);
    if (launch(s, a) != cudaSuccess) return RMRTLB_ECUDA;
    s->cur = 1 - s->cur;
    ++s->step;
    if (s->check_every > 0 && s->step % s->check_every == 0)
      if (run_check(s, 0, nullptr, nullptr, true, true) != cudaSuccess) return RMRTLB_ECUDA;
  }
  return RMRTLB_OK;
}

int rmrtlb_moments(rmrtlb_t s, double* rho, double* u) {
  if (!s) return RMRTLB_EINVAL;
  if (!rho && !u) return RMRTLB_OK;
  const size_t N = s->k.N;
  const bool rdev = !rho || is_device_ptr(rho);
  const bool udev = !u || is_device_ptr(u);
  double* r = rho ? (rdev ? rho : stage_ptr(s)) : nullptr;
  double* uu = u ? (udev ? u : stage_ptr(s) + N) : nullptr;
  if (run_check(s, 1, r, uu, false, false) != cudaSuccess) return RMRTLB_ECUDA;
  if (!rdev && cudaMemcpyAsync(rho, r, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  if (!udev && cudaMemcpyAsync(u, uu, s->k.d * N * sizeof(double), cudaMemcpyDeviceToHost, s->stream) !=
                   cudaSuccess)
    return RMRTLB_ECUDA;
  if ((!rdev || !udev) && cudaStreamSynchronize(s->stream) != cudaSuccess) return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

int rmrtlb_stats(rmrtlb_t s, double out[8]) {
  if (!s || !out) return RMRTLB_EINVAL;
  if (run_check(s, 1, nullptr, nullptr, true, false) != cudaSuccess) return RMRTLB_ECUDA;
  return read_slot(s, 1, out);
}

int rmrtlb_last_check(rmrtlb_t s, double out[8]) {
  if (!s || !out) return RMRTLB_EINVAL;
  if (!s->slot_valid[0]) {
    for (int i = 0; i < 8; ++i) out[i] = 0.0;
    out[5] = -1.0;
    out[6] = -1.0;
    return RMRTLB_OK;
  }
  return read_slot(s, 0, out);
}

}  // extern "C"
