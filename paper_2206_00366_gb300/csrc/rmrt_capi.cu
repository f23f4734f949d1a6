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
#include "rmrt_host.h"
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
using namespace rmrt::host;

namespace {

constexpr int kSlots = 2;          // 0: periodic check in rmrtlb_step, 1: rmrtlb_stats
constexpr int kInteriorMinPlanes = 5;   // rmrtlb_step_interior steps planes 2 .. n - 3 when n >= 5
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

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
  size_t fA, fB, stage, uprev, partials, stats, flags, hist, total, nblk;
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
  L.hist = L.flags + align_up(kSlots * sizeof(int));
  // B(t - dt) of the simplified NCDE, d planes in the compute type
  L.total = L.hist + align_up(d * N * (st == RMRTLB_ST_F64 ? sizeof(double) : sizeof(float)));
  return L;
}

bool valid_dims(int lat, int nx, int ny, int nz) {
  if (lat < 0 || lat > 4 || nx < 1 || ny < 1 || nz < 1) return false;
  if (lattice_d(lat) == 2 && nz != 1) return false;
  if (ny > 65535 || nz > 65535) return false;             // grid.y, grid.z limits
  const double N = double(nx) * ny * nz;
  return N * lattice_q(lat) < 9.0e18 && N < 2147483647.0;
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
  int quads;          // four nodes per thread (16-bit storage, nx % 4 == 0)
  bool interior_done; // rmrtlb_step_interior has stepped planes 2 .. n - 3 of the current step
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
  static const Fn table[5][5] = {
      {launch_d2q9_f64, launch_d2q9_f32, launch_d2q9_f16, launch_d2q9_bf16, launch_d2q9_e3m12},
      {launch_d3q19_f64, launch_d3q19_f32, launch_d3q19_f16, launch_d3q19_bf16, launch_d3q19_e3m12},
      {launch_d3q27_f64, launch_d3q27_f32, launch_d3q27_f16, launch_d3q27_bf16, launch_d3q27_e3m12},
      {launch_d2q5_f64, launch_d2q5_f32, launch_d2q5_f16, launch_d2q5_bf16, launch_d2q5_e3m12},
      {launch_d3q7_f64, launch_d3q7_f32, launch_d3q7_f16, launch_d3q7_bf16, launch_d3q7_e3m12}};
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

// ------------------------------------------------------------------ slab faces
// The axis along which a grid is cut into slabs: y on rD2Q9 / rD2Q5, z on
// the 3-D lattices.  The populations that cross a face are those with
// e_axis = +1 (going up) or -1 (going down), in increasing j.
int slab_axis(const rmrtlb_solver* s) { return s->k.d == 2 ? 1 : 2; }

int crossing(const rmrtlb_solver* s, int sign, int* dirs) {
  int n = 0;
  for (int j = 0; j < s->k.q; ++j) {
    int e[3];
    lattice_dir(s->k.lat, j, e);
    if (e[slab_axis(s)] == sign) dirs[n++] = j;
  }
  return n;
}

// Elements of one plane normal to the slab axis, and the offset of plane i.
size_t plane_elems(const rmrtlb_solver* s) {
  return s->k.d == 2 ? size_t(s->k.nx) : size_t(s->k.nx) * s->k.ny;
}

struct FaceCopy {
  int dirs[9];        // crossing directions
  int n;              // their count
  size_t off;         // element offset of the face plane inside a direction's plane
};

// Gather (to_buf) or scatter one face: buf[k * P + i] <-> f[dirs[k] * N + off + i].
template <typename E>
__global__ void face_kernel(E* __restrict__ f, E* __restrict__ buf, FaceCopy fc, size_t N, size_t P, int to_buf) {
  const size_t total = size_t(fc.n) * P;
  for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
    const size_t k = t / P, i = t - k * P;
    E* cell = f + size_t(fc.dirs[k]) * N + fc.off + i;
    if (to_buf) buf[t] = *cell;
    else *cell = buf[t];
  }
}

cudaError_t face_copy(rmrtlb_solver* s, int sign, void* buf, bool to_buf) {
  FaceCopy fc;
  fc.n = crossing(s, sign, fc.dirs);
  const size_t P = plane_elems(s);
  // up (+1): the last plane; down (-1): the first
  const size_t nplanes = s->k.d == 2 ? size_t(s->k.ny) : size_t(s->k.nz);
  fc.off = sign > 0 ? (nplanes - 1) * P : 0;
  const size_t total = size_t(fc.n) * P;
  const int threads = 256;
  const unsigned blocks = unsigned((total + threads - 1) / threads < 4096 ? (total + threads - 1) / threads : 4096);
  void* f = pop_ptr(s, s->cur);
  const size_t N = s->k.N;
  switch (storage_size(s->k.storage)) {
    case 8: face_kernel<unsigned long long><<<blocks, threads, 0, s->stream>>>(
        static_cast<unsigned long long*>(f), static_cast<unsigned long long*>(buf), fc, N, P, to_buf); break;
    case 4: face_kernel<unsigned><<<blocks, threads, 0, s->stream>>>(
        static_cast<unsigned*>(f), static_cast<unsigned*>(buf), fc, N, P, to_buf); break;
    default: face_kernel<unsigned short><<<blocks, threads, 0, s->stream>>>(
        static_cast<unsigned short*>(f), static_cast<unsigned short*>(buf), fc, N, P, to_buf); break;
  }
  return cudaGetLastError();
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
    case RMRTLB_ETIMEOUT: return "a bounded device-side wait gave up";
    default: return "unknown status";
  }
}

int rmrtlb_lattice_info(int lattice, int* q, int* d, int* e) {
  if (lattice < 0 || lattice > 4) return RMRTLB_EINVAL;
  if (q) *q = lattice_q(lattice);
  if (d) *d = lattice_d(lattice);
  if (e)
    for (int j = 0; j < lattice_q(lattice); ++j) lattice_dir(lattice, j, e + 3 * j);
  return RMRTLB_OK;
}

int rmrtlb_workspace_bytes(int lattice, int nx, int ny, int nz, int storage, size_t* bytes) {
  if (!bytes || !valid_dims(lattice, nx, ny, nz) || storage < 0 || storage > 4) return RMRTLB_EINVAL;
  *bytes = make_layout(lattice, nx, ny, nz, storage).total;
  return RMRTLB_OK;
}

int rmrtlb_create(rmrtlb_t* solver, int lattice, int nx, int ny, int nz, double dx, double dy, double dz,
                  double dt, const rmrtlb_params* params, int eq_kind, int basis, int storage, void* workspace,
                  size_t workspace_bytes, void* stream) {
  if (!solver || !params || !valid_dims(lattice, nx, ny, nz)) return RMRTLB_EINVAL;
  *solver = nullptr;
  if (eq_kind < 0 || eq_kind > 5 || basis < 0 || basis > 3 || storage < 0 || storage > 4) return RMRTLB_EINVAL;
  if (!(dt > 0) || !(dx > 0) || !(dy > 0) || (lattice_d(lattice) == 3 && !(dz > 0))) return RMRTLB_EINVAL;
  if (!workspace || (reinterpret_cast<size_t>(workspace) % kAlign) != 0) return RMRTLB_EINVAL;
  const Layout L = make_layout(lattice, nx, ny, nz, storage);
  if (workspace_bytes < L.total) return RMRTLB_ENOMEM;

  Consts k;
  const int rc = make_consts(k, lattice, nx, ny, nz, dx, dy, dz, dt, *params, eq_kind, basis, storage);
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
  s->kp64.hist = reinterpret_cast<double*>(s->ws + L.hist);
  s->kp32.hist = reinterpret_cast<float*>(s->ws + L.hist);
  s->kp64.hist_fresh = s->kp32.hist_fresh = 1;
  s->kp64.node_base = s->kp32.node_base = unsigned((unsigned long long)params->node_offset);
  s->check_every = params->check_every;
  s->pairs = (nx % 2 == 0) && !axis_lattice(lattice) && !simple_ncde(eq_kind);
  s->quads = s->pairs && nx % 4 == 0 &&
             (storage == RMRTLB_ST_F16 || storage == RMRTLB_ST_BF16 || storage == RMRTLB_ST_E3M12);
  s->interior_done = false;
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
  s->interior_done = false;
  s->kp64.hist_fresh = s->kp32.hist_fresh = 1;
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
  s->interior_done = false;
  s->kp64.hist_fresh = s->kp32.hist_fresh = 1;
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

}  // extern "C"

namespace {

// Extent of the slab axis (y on the 2-D lattices, z on the 3-D ones).
int axis_planes(const rmrtlb_solver* s) { return s->k.d == 2 ? s->k.ny : s->k.nz; }

// The step kernel over planes [first, first + count) of the slab axis:
// reads the current lattice, writes the other one.
cudaError_t launch_step_planes(rmrtlb_solver* s, int first, int count) {
  if (count <= 0) return cudaSuccess;
  LaunchArgs a = base_args(s, OP_STEP);
  if (s->quads) {
    const int quarter = s->k.nx / 4;
    const int bx = block_x(quarter);
    a.quads = 1;
    a.block = dim3(bx, 1, 1);
    a.grid = dim3((quarter + bx - 1) / bx, s->k.ny, s->k.nz);
  } else if (s->pairs) {
    const int half = s->k.nx / 2;
    const int bx = block_x(half);
    a.pairs = 1;
    a.block = dim3(bx, 1, 1);
    a.grid = dim3((half + bx - 1) / bx, s->k.ny, s->k.nz);
  }
  a.fin = pop_ptr(s, s->cur);
  a.fout = pop_ptr(s, 1 - s->cur);
  if (s->k.d == 2) a.grid.y = unsigned(count);
  else a.grid.z = unsigned(count);
  // seed of the stochastic rounding of 16-bit stores: a function of the
  // step index only, so a run is reproducible
  s->kp32.seed = unsigned((unsigned long long)s->step * 0x9E3779B97F4A7C15ull >> 32);
  s->kp64.plane0 = s->kp32.plane0 = first;
  const cudaError_t e = launch(s, a);   // the parameters are copied at launch
  s->kp64.plane0 = s->kp32.plane0 = 0;
  return e;
}

// Completes a step whose planes have all been stepped: swaps the lattices,
// advances the counter, runs the periodic check when one is due.
int finish_step(rmrtlb_solver* s) {
  s->kp64.hist_fresh = s->kp32.hist_fresh = 0;
  s->cur = 1 - s->cur;
  ++s->step;
  s->interior_done = false;
  if (s->check_every > 0 && s->step % s->check_every == 0)
    if (run_check(s, 0, nullptr, nullptr, true, true) != cudaSuccess) return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

}  // namespace

extern "C" {

int rmrtlb_step(rmrtlb_t s, int n) {
  if (!s || n < 0) return RMRTLB_EINVAL;
  for (int i = 0; i < n; ++i) {
    const int planes = axis_planes(s);
    // a step begun by rmrtlb_step_interior is completed first
    if (s->interior_done) {
      if (launch_step_planes(s, 0, 2) != cudaSuccess || launch_step_planes(s, planes - 2, 2) != cudaSuccess)
        return RMRTLB_ECUDA;
    } else if (launch_step_planes(s, 0, planes) != cudaSuccess) {
      return RMRTLB_ECUDA;
    }
    const int rc = finish_step(s);
    if (rc != RMRTLB_OK) return rc;
  }
  return RMRTLB_OK;
}

int rmrtlb_step_interior(rmrtlb_t s) {
  if (!s || s->interior_done) return RMRTLB_EINVAL;
  const int planes = axis_planes(s);
  if (planes < kInteriorMinPlanes) return RMRTLB_OK;   // every plane is a boundary plane
  if (launch_step_planes(s, 2, planes - 4) != cudaSuccess) return RMRTLB_ECUDA;
  s->interior_done = true;
  return RMRTLB_OK;
}

int rmrtlb_step_boundary(rmrtlb_t s) { return rmrtlb_step(s, 1); }

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

int rmrtlb_stress(rmrtlb_t s, double* stress, double* strain) {
  if (!s) return RMRTLB_EINVAL;
  if (s->k.kind != RMRTLB_EQ_NSE && s->k.kind != RMRTLB_EQ_NSE_HELUO) return RMRTLB_EINVAL;
  if ((stress && !is_device_ptr(stress)) || (strain && !is_device_ptr(strain))) return RMRTLB_EINVAL;
  if (!stress && !strain) return RMRTLB_OK;
  LaunchArgs a = base_args(s, OP_STRESS);
  a.fin = pop_ptr(s, s->cur);
  a.stress = stress;
  a.strain = strain;
  return launch(s, a) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
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

int rmrtlb_check(rmrtlb_t s) {
  if (!s) return RMRTLB_EINVAL;
  return run_check(s, 0, nullptr, nullptr, true, true) == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA;
}

int rmrtlb_check_sums(rmrtlb_t s, double out[8]) {
  if (!s || !out) return RMRTLB_EINVAL;
  for (int i = 0; i < 8; ++i) out[i] = 0.0;
  if (!s->slot_valid[0]) {
    out[6] = -1.0;
    return RMRTLB_OK;
  }
  double raw[8];
  int flags = 0;
  if (cudaMemcpyAsync(raw, s->ws + s->L.stats, sizeof(raw), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(&flags, s->ws + s->L.flags, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  out[0] = double(s->k.N) * s->k.rho0 + raw[0];
  out[1] = raw[1]; out[2] = raw[2]; out[3] = raw[3];
  out[4] = raw[4];
  out[5] = s->slot_prev[0] ? raw[5] : -1.0;
  out[6] = raw[6];
  out[7] = double(flags);
  return RMRTLB_OK;
}

int rmrtlb_halo_bytes(rmrtlb_t s, size_t* bytes) {
  if (!s || !bytes) return RMRTLB_EINVAL;
  int dirs[9];
  *bytes = size_t(crossing(s, +1, dirs)) * plane_elems(s) * storage_size(s->k.storage);
  return RMRTLB_OK;
}

int rmrtlb_halo_pack(rmrtlb_t s, void* up, void* down) {
  if (!s || !up || !down || !is_device_ptr(up) || !is_device_ptr(down)) return RMRTLB_EINVAL;
  if (face_copy(s, +1, up, true) != cudaSuccess || face_copy(s, -1, down, true) != cudaSuccess)
    return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

int rmrtlb_halo_unpack(rmrtlb_t s, const void* from_below, const void* from_above) {
  if (!s || !from_below || !from_above || !is_device_ptr(from_below) || !is_device_ptr(from_above))
    return RMRTLB_EINVAL;
  if (face_copy(s, +1, const_cast<void*>(from_below), false) != cudaSuccess ||
      face_copy(s, -1, const_cast<void*>(from_above), false) != cudaSuccess)
    return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ checkpoint / resume
// A state blob: a header (format, grid, storage, basis, kind, the step
// counter and check bookkeeping, and every derived constant of the step as
// a fingerprint of the parameters), then the raw population codes of the
// current lattice, the residual snapshot (when a check has written one),
// the simplified NCDE's B(t - dt) planes (that kind only), and the periodic
// check's stats and flag words.  The codes are copied as stored, so a
// resumed run draws the same stochastic-rounding bits and is bitwise
// identical to an uninterrupted one.
namespace {

constexpr int kFingerprint = 80;

struct StateHeader {
  char magic[8];
  unsigned version, header_bytes;
  int lattice, nx, ny, nz, storage, basis, eq_kind, has_prev;
  long long step;
  int hist_fresh, slot_valid, slot_prev;
  unsigned node_base;                  // rmrtlb_params.node_offset: where the rounding bits are drawn
  long long slot_step;
  double fp[kFingerprint];
  unsigned long long pop_bytes, prev_bytes, hist_bytes, stats_bytes, flags_bytes;
};
const char kStateMagic[8] = {'R', 'M', 'R', 'T', 'L', 'B', 'S', '1'};

void fingerprint(const Consts& k, double fp[kFingerprint]) {
  int i = 0;
  for (int a = 0; a < 3; ++a) fp[i++] = k.c[a];
  fp[i++] = k.cs2; fp[i++] = k.dt; fp[i++] = k.rho0; fp[i++] = k.source;
  for (int j = 0; j < 27; ++j) fp[i++] = k.w[j];
  fp[i++] = k.s0;
  for (int a = 0; a < 3; ++a) fp[i++] = k.s1[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) fp[i++] = k.s2[a][b];
  for (int a = 0; a < 3; ++a) fp[i++] = k.soff[a];
  fp[i++] = k.sfree;
  for (int a = 0; a < 3; ++a) { fp[i++] = k.ss[a]; fp[i++] = k.sb[a]; fp[i++] = k.force[a]; fp[i++] = k.adv[a]; }
  fp[i++] = double(k.st_shift);
  fp[i++] = double(k.forced);
  while (i < kFingerprint) fp[i++] = 0.0;
}

size_t round16(size_t v) { return (v + 15) / 16 * 16; }

// Section sizes of this solver's state.
void state_sections(const rmrtlb_solver* s, size_t& pop, size_t& prev, size_t& hist, size_t& stats, size_t& flags) {
  const size_t ct = s->k.storage == RMRTLB_ST_F64 ? sizeof(double) : sizeof(float);
  pop = size_t(s->k.q) * s->k.N * storage_size(s->k.storage);
  prev = s->has_prev ? size_t(s->k.d) * s->k.N * ct : 0;
  hist = simple_ncde(s->k.kind) ? size_t(s->k.d) * s->k.N * ct : 0;
  stats = 8 * sizeof(double);
  flags = sizeof(int);
}

}  // namespace

int rmrtlb_state_bytes(rmrtlb_t s, size_t* bytes) {
  if (!s || !bytes) return RMRTLB_EINVAL;
  size_t pop, prev, hist, stats, flags;
  state_sections(s, pop, prev, hist, stats, flags);
  *bytes = round16(sizeof(StateHeader)) + round16(pop) + round16(prev) + round16(hist) + round16(stats) +
           round16(flags);
  return RMRTLB_OK;
}

int rmrtlb_save_state(rmrtlb_t s, void* dst, size_t bytes) {
  size_t need = 0;
  if (!s || !dst || rmrtlb_state_bytes(s, &need) != RMRTLB_OK || bytes < need) return RMRTLB_EINVAL;
  size_t pop, prev, hist, stats, flags;
  state_sections(s, pop, prev, hist, stats, flags);
  StateHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kStateMagic, 8);
  h.version = 1;
  h.header_bytes = unsigned(sizeof(StateHeader));
  h.lattice = s->k.lat; h.nx = s->k.nx; h.ny = s->k.ny; h.nz = s->k.nz;
  h.storage = s->k.storage; h.basis = s->k.central; h.eq_kind = s->k.kind;
  h.has_prev = s->has_prev ? 1 : 0;
  h.step = s->step;
  h.hist_fresh = s->kp32.hist_fresh;
  h.slot_valid = s->slot_valid[0] ? 1 : 0;
  h.slot_prev = s->slot_prev[0] ? 1 : 0;
  h.slot_step = s->slot_step[0];
  h.node_base = s->kp32.node_base;
  fingerprint(s->k, h.fp);
  h.pop_bytes = pop; h.prev_bytes = prev; h.hist_bytes = hist; h.stats_bytes = stats; h.flags_bytes = flags;
  char* d = static_cast<char*>(dst);
  size_t off = 0;
  static const char zeros[16] = {0};
  // each section, then zeros up to its 16-byte boundary (a blob is fully defined)
  auto put = [&](const void* src, size_t n) {
    bool ok = n == 0 || cudaMemcpyAsync(d + off, src, n, cudaMemcpyDefault, s->stream) == cudaSuccess;
    if (round16(n) > n)
      ok = ok && cudaMemcpyAsync(d + off + n, zeros, round16(n) - n, cudaMemcpyDefault, s->stream) == cudaSuccess;
    off += round16(n);
    return ok;
  };
  const bool ok = put(&h, sizeof(h)) && put(pop_ptr(s, s->cur), pop) && put(s->ws + s->L.uprev, prev) &&
                  put(s->ws + s->L.hist, hist) && put(s->ws + s->L.stats, stats) && put(s->ws + s->L.flags, flags);
  // the header lives on this stack frame: the copies end before returning
  if (cudaStreamSynchronize(s->stream) != cudaSuccess || !ok) return RMRTLB_ECUDA;
  return RMRTLB_OK;
}

int rmrtlb_load_state(rmrtlb_t s, const void* src, size_t bytes) {
  if (!s || !src || bytes < sizeof(StateHeader)) return RMRTLB_EINVAL;
  StateHeader h;
  if (cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDefault, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return RMRTLB_ECUDA;
  double fp[kFingerprint];
  fingerprint(s->k, fp);
  if (memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1 || h.header_bytes != sizeof(StateHeader) ||
      h.lattice != s->k.lat || h.nx != s->k.nx || h.ny != s->k.ny || h.nz != s->k.nz ||
      h.storage != s->k.storage || h.basis != s->k.central || h.eq_kind != s->k.kind ||
      memcmp(h.fp, fp, sizeof(fp)) != 0 || h.node_base != s->kp32.node_base || h.step < 0)
    return RMRTLB_EINVAL;
  // the section sizes this solver expects with the blob's snapshot flag
  const bool had_prev = s->has_prev;
  s->has_prev = h.has_prev != 0;
  size_t pop, prev, hist, stats, flags, need = 0;
  state_sections(s, pop, prev, hist, stats, flags);
  rmrtlb_state_bytes(s, &need);
  s->has_prev = had_prev;
  if (bytes < need || h.pop_bytes != pop || h.prev_bytes != prev || h.hist_bytes != hist || h.stats_bytes != stats ||
      h.flags_bytes != flags)
    return RMRTLB_EINVAL;
  const char* p = static_cast<const char*>(src) + round16(sizeof(StateHeader));
  auto get = [&](void* dst, size_t n) {
    const bool ok = n == 0 || cudaMemcpyAsync(dst, p, n, cudaMemcpyDefault, s->stream) == cudaSuccess;
    p += round16(n);
    return ok;
  };
  const bool ok = get(pop_ptr(s, 0), pop) && get(s->ws + s->L.uprev, prev) && get(s->ws + s->L.hist, hist) &&
                  get(s->ws + s->L.stats, stats) && get(s->ws + s->L.flags, flags);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess || !ok) return RMRTLB_ECUDA;
  s->cur = 0;
  s->interior_done = false;
  s->step = h.step;
  s->has_prev = h.has_prev != 0;
  s->kp64.hist_fresh = s->kp32.hist_fresh = h.hist_fresh;
  s->slot_valid[0] = h.slot_valid != 0;
  s->slot_prev[0] = h.slot_prev != 0;
  s->slot_step[0] = h.slot_step;
  return RMRTLB_OK;
}
