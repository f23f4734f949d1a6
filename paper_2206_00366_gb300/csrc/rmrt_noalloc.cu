// Allocation-free FP64 population totals (rmrtlb_population_totals_noalloc).
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (a framework's caching allocator or a fixed pool sized in
// advance), or code that must not let an allocation synchronise the device
// in the middle of its stream work.  For them this file keeps the scratch of
// the deterministic two-level FP64 reduction in a file-scope device array of
// fixed size instead of in a caller workspace.  The array exists once per
// GPU that loads the library and lives until the process exits.
//
// The caller passes the populations (device memory) and the output; nothing
// here allocates.  Every call shares the one array: two calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// it and may return wrong totals.  Calls issued on one stream are ordered.
// No slot needs clearing: each block writes its own partial row before the
// second kernel, in the same call, reads it.
#include <mutex>

#include "../../include/rmrtlb.h"
#include "rmrt_device.cuh"

namespace rmrt {

constexpr int NA_THREADS = 256;
constexpr int NA_NODES_PER_BLOCK = 16384;                 // 64 nodes per thread
constexpr int NA_MAX_BLOCKS = 4096;
constexpr long long NA_MAX_NODES = (long long)NA_MAX_BLOCKS * NA_NODES_PER_BLOCK;
static_assert(NA_MAX_NODES == RMRTLB_NOALLOC_MAX_NODES, "header limit out of date");

// NA_MAX_BLOCKS partial rows of 8 doubles, then 8 doubles for the result.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS * 8 + 8];

// Per-block sums over a contiguous chunk of nodes: [0] sum f, [1..3] sum c f,
// [4] sum |sum c f|^2 / (2 sum f).  Canonical FP64 populations, q planes.
template <int LAT>
__global__ void __launch_bounds__(NA_THREADS) totals_kernel(const double* __restrict__ f, size_t N, double c0,
                                                            double c1, double c2, double* __restrict__ scratch) {
  using L = Lat<LAT>;
  const double c[3] = {c0, c1, c2};
  double acc[5] = {0, 0, 0, 0, 0};
  const size_t begin = size_t(blockIdx.x) * NA_NODES_PER_BLOCK;
  const size_t end = begin + NA_NODES_PER_BLOCK < N ? begin + NA_NODES_PER_BLOCK : N;
  for (size_t n = begin + threadIdx.x; n < end; n += NA_THREADS) {
    double m0 = 0, m1[3] = {0, 0, 0};
    static_for<L::Q>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int ex = L::EX[j], ey = L::EY[j], ez = L::EZ[j];
      const double v = f[size_t(j) * N + n];
      m0 += v;
      if (ex) m1[0] += ex * c[0] * v;
      if (ey) m1[1] += ey * c[1] * v;
      if (ez) m1[2] += ez * c[2] * v;
    });
    acc[0] += m0;
    acc[1] += m1[0]; acc[2] += m1[1]; acc[3] += m1[2];
    if (m0 != 0.0) acc[4] += 0.5 * (m1[0] * m1[0] + m1[1] * m1[1] + m1[2] * m1[2]) / m0;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  __shared__ double sm[NA_THREADS / 32][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 5; ++k) sm[warp][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0;
    for (int w = 0; w < NA_THREADS / 32; ++w) s += sm[w][threadIdx.x];
    scratch[size_t(blockIdx.x) * 8 + threadIdx.x] = s;
  }
}

// Fixed-order sum of the nblk partial rows into out[0..4].
__global__ void __launch_bounds__(NA_THREADS) totals_finalize(const double* __restrict__ scratch, int nblk,
                                                              double* __restrict__ out) {
  __shared__ double sm[5][NA_THREADS];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nblk; i += NA_THREADS)
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += scratch[size_t(i) * 8 + k];
#pragma unroll
  for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = sm[threadIdx.x][0];
}

}  // namespace rmrt

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.  The array's name in host code is a
// host-side stand-in, never a device address, so kernels only ever get the
// pointer returned here.
cudaError_t scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, rmrt::g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<double*>(g_scratch_ptr[dev]);
  return cudaSuccess;
}

enum Where { HOST_MEMORY, THIS_DEVICE, OTHER_DEVICE };

// Where a pointer lives relative to the current device dev: device memory
// of dev and managed memory (the kernels reach both from dev) are
// THIS_DEVICE, device memory of another GPU is OTHER_DEVICE, pageable and
// pinned host memory are HOST_MEMORY.
Where where_is(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();   // the query's own error: unregistered host memory on old runtimes
    return HOST_MEMORY;
  }
  if (at.type == cudaMemoryTypeManaged) return THIS_DEVICE;
  if (at.type == cudaMemoryTypeDevice) return at.device == dev ? THIS_DEVICE : OTHER_DEVICE;
  return HOST_MEMORY;
}

}  // namespace

extern "C" int rmrtlb_population_totals_noalloc(int lattice, int nx, int ny, int nz, double dx, double dy,
                                                double dz, double dt, const double* f, double* out,
                                                void* stream) {
  using namespace rmrt;
  if (lattice < 0 || lattice > 2 || nx < 1 || ny < 1 || nz < 1 || !f || !out) return RMRTLB_EINVAL;
  if (lattice == RMRTLB_D2Q9 && nz != 1) return RMRTLB_EINVAL;
  if (!(dt > 0) || !(dx > 0) || !(dy > 0) || (lattice != RMRTLB_D2Q9 && !(dz > 0))) return RMRTLB_EINVAL;
  const long long N = (long long)nx * ny * nz;
  if (N > NA_MAX_NODES) return RMRTLB_ETOOBIG;
  // an error left pending by earlier work is not ours: report it, keep it
  if (cudaPeekAtLastError() != cudaSuccess) return RMRTLB_ECUDA;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RMRTLB_ECUDA;
  if (where_is(f, dev) != THIS_DEVICE) return RMRTLB_EINVAL;
  const Where out_at = where_is(out, dev);
  if (out_at == OTHER_DEVICE) return RMRTLB_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (out_at == HOST_MEMORY) {
    // a host out needs a copy and a synchronisation, neither of which a capture may hold
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return RMRTLB_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return RMRTLB_EINVAL;
  }
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) return RMRTLB_ECUDA;
  const int nblk = int((N + NA_NODES_PER_BLOCK - 1) / NA_NODES_PER_BLOCK);
  const double cx = dx / dt, cy = dy / dt, cz = lattice == RMRTLB_D2Q9 ? 0.0 : dz / dt;
  switch (lattice) {
    case RMRTLB_D2Q9: totals_kernel<LAT_D2Q9><<<nblk, NA_THREADS, 0, s>>>(f, size_t(N), cx, cy, cz, scratch); break;
    case RMRTLB_D3Q19: totals_kernel<LAT_D3Q19><<<nblk, NA_THREADS, 0, s>>>(f, size_t(N), cx, cy, cz, scratch); break;
    default: totals_kernel<LAT_D3Q27><<<nblk, NA_THREADS, 0, s>>>(f, size_t(N), cx, cy, cz, scratch); break;
  }
  if (cudaGetLastError() != cudaSuccess) return RMRTLB_ECUDA;
  const bool out_dev = out_at == THIS_DEVICE;
  double* result = out_dev ? out : scratch + size_t(NA_MAX_BLOCKS) * 8;
  totals_finalize<<<1, NA_THREADS, 0, s>>>(scratch, nblk, result);
  if (cudaGetLastError() != cudaSuccess) return RMRTLB_ECUDA;
  if (!out_dev) {
    if (cudaMemcpyAsync(out, result, 5 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return RMRTLB_ECUDA;
  }
  return RMRTLB_OK;
}
