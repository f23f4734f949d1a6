// Kernels of the warm-start network (include/rmrtlb_cnn.h): 3 x 3 x 3
// convolution forward and backward, MSE, Adam, input features, trilinear
// upsampling.  BF16 activations and weights, FP32 accumulation.
//
// The convolutions run on the FP32 pipes: one thread per output voxel and
// group of up to 8 output channels, the block's weight slice staged once
// in shared memory as FP32, input rows read as 16-byte vectors (8 BF16
// channels).  Every reduction over voxels is done in a fixed order (per
// block partials, then a fixed-order sum), so results are deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/rmrtlb.h"
#include "../../include/rmrtlb_cnn.h"

namespace {

constexpr int kThreads = 128;
constexpr int kWeightChunk = 4096;   // voxels per partial sum of the weight gradient

struct Vol {
  int n, d, h, w;
  __host__ __device__ long long voxels() const { return (long long)n * d * h * w; }
};

__device__ __forceinline__ float bf2f(uint16_t b) { return __uint_as_float(uint32_t(b) << 16); }
__device__ __forceinline__ uint16_t f2bf(float f) {
  const __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t*>(&h);
}
__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

// Coordinates of voxel index v (x fastest) and the index of its neighbour at
// offset (dz, dy, dx), or -1 outside the volume.
struct VoxCoord {
  int s, z, y, x;
};
__device__ __forceinline__ VoxCoord coord_of(long long v, const Vol& g) {
  VoxCoord c;
  c.x = int(v % g.w);
  long long r = v / g.w;
  c.y = int(r % g.h);
  r /= g.h;
  c.z = int(r % g.d);
  c.s = int(r / g.d);
  return c;
}
__device__ __forceinline__ long long neighbour(const VoxCoord& c, int dz, int dy, int dx, const Vol& g) {
  const int z = c.z + dz, y = c.y + dy, x = c.x + dx;
  if (unsigned(z) >= unsigned(g.d) || unsigned(y) >= unsigned(g.h) || unsigned(x) >= unsigned(g.w)) return -1;
  return (((long long)c.s * g.d + z) * g.h + y) * g.w + x;
}

// ------------------------------------------------------------------ forward
// grid (ceil(V / 128), COUT / G); thread: one voxel, output channels
// [G * blockIdx.y, G * blockIdx.y + G), G = min(8, COUT).
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) conv_fwd_kernel(Vol g, const uint16_t* __restrict__ x,
                                                            const uint16_t* __restrict__ wt,
                                                            const float* __restrict__ bias, int apply_silu,
                                                            float* __restrict__ z, uint16_t* __restrict__ a) {
  constexpr int G = COUT < 8 ? COUT : 8;
  __shared__ float ws[27 * CIN * G];
  const int co0 = blockIdx.y * G;
  for (int i = threadIdx.x; i < 27 * CIN * G; i += kThreads) {
    const int gg = i % G, tc = i / G;   // tc = t * CIN + ci
    ws[i] = bf2f(wt[size_t(tc) * COUT + co0 + gg]);
  }
  __syncthreads();
  const long long v = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (v >= g.voxels()) return;
  const VoxCoord c = coord_of(v, g);
  float acc[G];
#pragma unroll
  for (int k = 0; k < G; ++k) acc[k] = bias[co0 + k];
  for (int t = 0; t < 27; ++t) {
    const long long nb = neighbour(c, t / 9 - 1, (t / 3) % 3 - 1, t % 3 - 1, g);
    if (nb < 0) continue;
    const uint4* src = reinterpret_cast<const uint4*>(x + nb * CIN);
#pragma unroll
    for (int q = 0; q < CIN / 8; ++q) {
      const uint4 pk = __ldg(src + q);
      const uint32_t wd[4] = {pk.x, pk.y, pk.z, pk.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float xv = bf2f(uint16_t(wd[e >> 1] >> (16 * (e & 1))));
        const float* wr = ws + (t * CIN + q * 8 + e) * G;
#pragma unroll
        for (int k = 0; k < G; ++k) acc[k] = fmaf(xv, wr[k], acc[k]);
      }
    }
  }
  if (z) {
    float4* zo = reinterpret_cast<float4*>(z + v * COUT + co0);
#pragma unroll
    for (int k = 0; k < G / 4; ++k) zo[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
  }
  if (a) {
    uint32_t pk[G / 2];
#pragma unroll
    for (int k = 0; k < G / 2; ++k) {
      float p0 = acc[2 * k], p1 = acc[2 * k + 1];
      if (apply_silu) {
        p0 *= sigm(p0);
        p1 *= sigm(p1);
      }
      pk[k] = uint32_t(f2bf(p0)) | (uint32_t(f2bf(p1)) << 16);
    }
    uint32_t* ao = reinterpret_cast<uint32_t*>(a + v * COUT + co0);
#pragma unroll
    for (int k = 0; k < G / 2; ++k) ao[k] = pk[k];
  }
}

// ------------------------------------------------------------------ backward data
// grid (ceil(V / 128), CIN / G); thread: one voxel, input channels
// [G * blockIdx.y, G * blockIdx.y + G).
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) conv_bwd_data_kernel(Vol g, const float* __restrict__ dy,
                                                                 const uint16_t* __restrict__ wt,
                                                                 const float* __restrict__ zin,
                                                                 float* __restrict__ dx) {
  constexpr int G = CIN < 8 ? CIN : 8;
  __shared__ float ws[27 * COUT * G];   // ws[(t * COUT + co) * G + k] = w[t, ci0 + k, co]
  const int ci0 = blockIdx.y * G;
  for (int i = threadIdx.x; i < 27 * COUT * G; i += kThreads) {
    const int k = i % G, tc = i / G, co = tc % COUT, t = tc / COUT;
    ws[i] = bf2f(wt[(size_t(t) * CIN + ci0 + k) * COUT + co]);
  }
  __syncthreads();
  const long long v = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (v >= g.voxels()) return;
  const VoxCoord c = coord_of(v, g);
  float acc[G];
#pragma unroll
  for (int k = 0; k < G; ++k) acc[k] = 0.0f;
  for (int t = 0; t < 27; ++t) {
    // dy at v - tap_t
    const long long nb = neighbour(c, 1 - t / 9, 1 - (t / 3) % 3, 1 - t % 3, g);
    if (nb < 0) continue;
    const float4* src = reinterpret_cast<const float4*>(dy + nb * COUT);
#pragma unroll
    for (int q = 0; q < COUT / 4; ++q) {
      const float4 d4 = __ldg(src + q);
      const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float* wr = ws + (t * COUT + q * 4 + e) * G;
#pragma unroll
        for (int k = 0; k < G; ++k) acc[k] = fmaf(dv[e], wr[k], acc[k]);
      }
    }
  }
  if (zin) {
    const float* zr = zin + v * CIN + ci0;
#pragma unroll
    for (int k = 0; k < G; ++k) {
      const float zz = zr[k], s = sigm(zz);
      acc[k] *= s * (1.0f + zz * (1.0f - s));
    }
  }
  float4* out = reinterpret_cast<float4*>(dx + v * CIN + ci0);
#pragma unroll
  for (int k = 0; k < G / 4; ++k) out[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
}

// ------------------------------------------------------------------ backward weight
// grid (chunks, 27): block (c, t) sums x[v + tap_t, ci] dy[v, co] over the
// chunk's voxels into part[(c * 27 + t) * CIN * COUT + ci * COUT + co]; the
// t = 13 (centre) block also writes the chunk's bias sums to
// bpart[c * COUT + co].  Voxels are staged 128 at a time in shared memory.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) conv_bwd_weight_kernel(Vol g, const uint16_t* __restrict__ x,
                                                              const float* __restrict__ dy,
                                                              float* __restrict__ part, float* __restrict__ bpart) {
  constexpr int NOUT = CIN * COUT, PER = (NOUT + 255) / 256, SUB = 128;
  __shared__ float xs[SUB][CIN];
  __shared__ float ds[SUB][COUT];
  const int t = blockIdx.y;
  const int dz = t / 9 - 1, dyo = (t / 3) % 3 - 1, dxo = t % 3 - 1;
  const long long V = g.voxels();
  const long long v0 = (long long)blockIdx.x * kWeightChunk;
  const long long v1 = v0 + kWeightChunk < V ? v0 + kWeightChunk : V;
  float acc[PER], bacc = 0.0f;
#pragma unroll
  for (int p = 0; p < PER; ++p) acc[p] = 0.0f;
  for (long long s0 = v0; s0 < v1; s0 += SUB) {
    __syncthreads();
    for (int i = threadIdx.x; i < SUB * CIN; i += 256) {
      const int vv = i / CIN, ci = i % CIN;
      const long long v = s0 + vv;
      float val = 0.0f;
      if (v < v1) {
        const long long nb = neighbour(coord_of(v, g), dz, dyo, dxo, g);
        if (nb >= 0) val = bf2f(x[nb * CIN + ci]);
      }
      xs[vv][ci] = val;
    }
    for (int i = threadIdx.x; i < SUB * COUT; i += 256) {
      const int vv = i / COUT, co = i % COUT;
      const long long v = s0 + vv;
      ds[vv][co] = v < v1 ? dy[v * COUT + co] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int o = threadIdx.x + 256 * p;
      if (o < NOUT) {
        const int ci = o / COUT, co = o % COUT;
        float s = acc[p];
        for (int vv = 0; vv < SUB; ++vv) s = fmaf(xs[vv][ci], ds[vv][co], s);
        acc[p] = s;
      }
    }
    if (t == 13 && threadIdx.x < COUT) {
      float s = bacc;
      for (int vv = 0; vv < SUB; ++vv) s += ds[vv][threadIdx.x];
      bacc = s;
    }
  }
  float* out = part + (size_t(blockIdx.x) * 27 + t) * NOUT;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int o = threadIdx.x + 256 * p;
    if (o < NOUT) out[o] = acc[p];
  }
  if (t == 13 && threadIdx.x < COUT) bpart[size_t(blockIdx.x) * COUT + threadIdx.x] = bacc;
}

// Fixed-order sum over chunks: out[i] = sum_c part[c * stride + i], i < n.
__global__ void sum_chunks_kernel(const float* __restrict__ part, int chunks, size_t stride, int n,
                                  float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int c = 0; c < chunks; ++c) s += part[size_t(c) * stride + i];
  out[i] = s;
}

// ------------------------------------------------------------------ loss, optimiser
constexpr int kMseBlocks = 1024;

__global__ void __launch_bounds__(256) mse_kernel(long long count, const float* __restrict__ y,
                                                  const float* __restrict__ t, float* __restrict__ dy,
                                                  double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  const float sc = float(2.0 / double(count));
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < count; i += (long long)gridDim.x * 256) {
    const float r = y[i] - t[i];
    dy[i] = sc * r;
    s += double(r) * double(r);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (int(threadIdx.x) < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) mse_final_kernel(const double* __restrict__ part, int n, long long count,
                                                        double* __restrict__ loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (int(threadIdx.x) < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / double(count);
}

__global__ void adam_kernel(long long count, float* __restrict__ p, uint16_t* __restrict__ pb,
                            const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = f2bf(pi);
  }
}

// ------------------------------------------------------------------ features, upsampling
__global__ void features_kernel(Vol g, const double* __restrict__ re, uint16_t* __restrict__ x) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.voxels()) return;
  const VoxCoord c = coord_of(v, g);
  const double xh = (c.x + 0.5) / g.w * 2.0 - 1.0, yh = (c.y + 0.5) / g.h * 2.0 - 1.0;
  const double zh = (c.z + 0.5) / g.d * 2.0 - 1.0, rh = (re[c.s] - 800.0) / 700.0;
  const double f[8] = {xh, yh, zh, rh, xh * zh, yh * zh, zh * zh, rh * zh};
  uint32_t pk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) pk[k] = uint32_t(f2bf(float(f[2 * k]))) | (uint32_t(f2bf(float(f[2 * k + 1]))) << 16);
  reinterpret_cast<uint4*>(x)[v] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}

struct UpArgs {
  int d, h, w, c, D, H, W;
  double scale[8], offset[8];
};

__device__ __forceinline__ void lin(int I, int N, int n, int& i0, int& i1, double& f) {
  double s = (I + 0.5) * double(n) / double(N) - 0.5;
  s = s < 0.0 ? 0.0 : (s > n - 1 ? double(n - 1) : s);
  i0 = int(floor(s));
  i1 = i0 + 1 < n ? i0 + 1 : n - 1;
  f = s - i0;
}

__global__ void upsample_kernel(UpArgs a, const float* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)a.D * a.H * a.W;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int X = int(i % a.W), Y = int((i / a.W) % a.H), Z = int(i / ((long long)a.W * a.H));
  int x0, x1, y0, y1, z0, z1;
  double fx, fy, fz;
  lin(X, a.W, a.w, x0, x1, fx);
  lin(Y, a.H, a.h, y0, y1, fy);
  lin(Z, a.D, a.d, z0, z1, fz);
  auto at = [&](int z, int y, int x, int k) -> double {
    return double(src[((size_t(z) * a.h + y) * a.w + x) * a.c + k]);
  };
  for (int k = 0; k < a.c; ++k) {
    // interpolate along x, then y, then z
    const double c00 = at(z0, y0, x0, k) * (1 - fx) + at(z0, y0, x1, k) * fx;
    const double c01 = at(z0, y1, x0, k) * (1 - fx) + at(z0, y1, x1, k) * fx;
    const double c10 = at(z1, y0, x0, k) * (1 - fx) + at(z1, y0, x1, k) * fx;
    const double c11 = at(z1, y1, x0, k) * (1 - fx) + at(z1, y1, x1, k) * fx;
    const double c0 = c00 * (1 - fy) + c01 * fy, c1 = c10 * (1 - fy) + c11 * fy;
    dst[size_t(k) * N + i] = a.offset[k] + a.scale[k] * (c0 * (1 - fz) + c1 * fz);
  }
}

__global__ void pack_kernel(long long n, int d, const double* __restrict__ rho, const double* __restrict__ u,
                            double rho0, double rs, double us, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 o;
  o.x = float((rho[i] - rho0) * rs);
  o.y = float(u[i] * us);
  o.z = float(u[n + i] * us);
  o.w = d == 3 ? float(u[2 * n + i] * us) : 0.0f;
  reinterpret_cast<float4*>(out)[i] = o;
}

bool aligned16(const void* p) { return p && (reinterpret_cast<size_t>(p) & 15) == 0; }
bool vol_ok(int n, int d, int h, int w) {
  return n > 0 && d > 0 && h > 0 && w > 0 && double(n) * d * h * w < 2147483647.0;
}
int status_of(cudaError_t e) { return e == cudaSuccess ? RMRTLB_OK : RMRTLB_ECUDA; }
unsigned blocks_for(long long items, int per) { return unsigned((items + per - 1) / per); }

template <int CIN, int COUT>
int fwd(Vol g, const uint16_t* x, const uint16_t* w, const float* b, int silu, float* z, uint16_t* a,
        cudaStream_t s) {
  constexpr int G = COUT < 8 ? COUT : 8;
  conv_fwd_kernel<CIN, COUT><<<dim3(blocks_for(g.voxels(), kThreads), COUT / G), kThreads, 0, s>>>(g, x, w, b, silu,
                                                                                                    z, a);
  return status_of(cudaGetLastError());
}

template <int CIN, int COUT>
int bwd_data(Vol g, const float* dy, const uint16_t* w, const float* zin, float* dx, cudaStream_t s) {
  constexpr int G = CIN < 8 ? CIN : 8;
  conv_bwd_data_kernel<CIN, COUT><<<dim3(blocks_for(g.voxels(), kThreads), CIN / G), kThreads, 0, s>>>(g, dy, w,
                                                                                                        zin, dx);
  return status_of(cudaGetLastError());
}

int chunks_of(Vol g) { return int((g.voxels() + kWeightChunk - 1) / kWeightChunk); }

template <int CIN, int COUT>
int bwd_weight(Vol g, const uint16_t* x, const float* dy, float* dw, float* db, float* scratch, cudaStream_t s) {
  const int chunks = chunks_of(g);
  float* part = scratch;
  float* bpart = scratch + size_t(chunks) * 27 * CIN * COUT;
  conv_bwd_weight_kernel<CIN, COUT><<<dim3(chunks, 27), 256, 0, s>>>(g, x, dy, part, bpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return RMRTLB_ECUDA;
  const int nw = 27 * CIN * COUT;
  sum_chunks_kernel<<<blocks_for(nw, 256), 256, 0, s>>>(part, chunks, size_t(nw), nw, dw);
  sum_chunks_kernel<<<1, 256, 0, s>>>(bpart, chunks, size_t(COUT), COUT, db);
  return status_of(cudaGetLastError());
}

}  // namespace

extern "C" {

int rmrtlb_conv3d_forward(int n, int d, int h, int w, int cin, int cout, const uint16_t* x, const uint16_t* weight,
                          const float* bias, int apply_silu, float* z, uint16_t* a, void* stream) {
  if (!vol_ok(n, d, h, w) || !aligned16(x) || !weight || !bias || (!z && !a)) return RMRTLB_EINVAL;
  if ((z && !aligned16(z)) || (a && (reinterpret_cast<size_t>(a) & 7))) return RMRTLB_EINVAL;
  const Vol g{n, d, h, w};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cin == 8 && cout == 32) return fwd<8, 32>(g, x, weight, bias, apply_silu, z, a, s);
  if (cin == 32 && cout == 32) return fwd<32, 32>(g, x, weight, bias, apply_silu, z, a, s);
  if (cin == 32 && cout == 4) return fwd<32, 4>(g, x, weight, bias, apply_silu, z, a, s);
  return RMRTLB_EINVAL;
}

int rmrtlb_conv3d_backward_data(int n, int d, int h, int w, int cin, int cout, const float* dy,
                                const uint16_t* weight, const float* z_in, float* dx, void* stream) {
  if (!vol_ok(n, d, h, w) || !aligned16(dy) || !weight || !aligned16(dx)) return RMRTLB_EINVAL;
  const Vol g{n, d, h, w};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cin == 32 && cout == 32) return bwd_data<32, 32>(g, dy, weight, z_in, dx, s);
  if (cin == 32 && cout == 4) return bwd_data<32, 4>(g, dy, weight, z_in, dx, s);
  return RMRTLB_EINVAL;
}

size_t rmrtlb_conv3d_backward_weight_scratch(int n, int d, int h, int w, int cin, int cout) {
  if (!vol_ok(n, d, h, w) || cin < 1 || cout < 1) return 0;
  const size_t chunks = size_t(chunks_of(Vol{n, d, h, w}));
  return (chunks * 27 * size_t(cin) * cout + chunks * cout) * sizeof(float);
}

int rmrtlb_conv3d_backward_weight(int n, int d, int h, int w, int cin, int cout, const uint16_t* x, const float* dy,
                                  float* dweight, float* dbias, void* scratch, size_t scratch_bytes, void* stream) {
  if (!vol_ok(n, d, h, w) || !x || !dy || !dweight || !dbias || !scratch) return RMRTLB_EINVAL;
  if (scratch_bytes < rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, cin, cout)) return RMRTLB_ENOMEM;
  const Vol g{n, d, h, w};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* sc = static_cast<float*>(scratch);
  if (cin == 8 && cout == 32) return bwd_weight<8, 32>(g, x, dy, dweight, dbias, sc, s);
  if (cin == 32 && cout == 32) return bwd_weight<32, 32>(g, x, dy, dweight, dbias, sc, s);
  if (cin == 32 && cout == 4) return bwd_weight<32, 4>(g, x, dy, dweight, dbias, sc, s);
  return RMRTLB_EINVAL;
}

int rmrtlb_mse(long long count, const float* y, const float* t, float* dy, double* loss, void* scratch,
               void* stream) {
  if (count < 1 || !y || !t || !dy || !loss || !scratch) return RMRTLB_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long want = (count + 255) / 256;
  const int blocks = int(want < kMseBlocks ? want : kMseBlocks);
  double* part = static_cast<double*>(scratch);
  mse_kernel<<<blocks, 256, 0, s>>>(count, y, t, dy, part);
  mse_final_kernel<<<1, 256, 0, s>>>(part, blocks, count, loss);
  return status_of(cudaGetLastError());
}

int rmrtlb_adam(long long count, float* param, uint16_t* param_bf16, const float* grad, float* m, float* v, int step,
                float lr, float beta1, float beta2, float eps, void* stream) {
  if (count < 1 || !param || !grad || !m || !v || step < 1) return RMRTLB_EINVAL;
  const float c1 = float(1.0 - pow(double(beta1), step)), c2 = float(1.0 - pow(double(beta2), step));
  const long long want = (count + 255) / 256;
  const unsigned blocks = unsigned(want < 4096 ? want : 4096);
  adam_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(count, param, param_bf16, grad, m, v, lr, beta1,
                                                                    beta2, eps, c1, c2);
  return status_of(cudaGetLastError());
}

int rmrtlb_cavity_features(int n, int d, int h, int w, const double* re, uint16_t* x, void* stream) {
  if (!vol_ok(n, d, h, w) || !re || !aligned16(x)) return RMRTLB_EINVAL;
  const Vol g{n, d, h, w};
  features_kernel<<<blocks_for(g.voxels(), 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(g, re, x);
  return status_of(cudaGetLastError());
}

int rmrtlb_upsample_fields(int d, int h, int w, int c, const float* src, int D, int H, int W, const double* scale,
                           const double* offset, double* dst, void* stream) {
  if (!vol_ok(1, d, h, w) || !vol_ok(1, D, H, W) || c < 1 || c > 8 || !src || !scale || !offset || !dst)
    return RMRTLB_EINVAL;
  UpArgs a;
  a.d = d; a.h = h; a.w = w; a.c = c; a.D = D; a.H = H; a.W = W;
  for (int k = 0; k < 8; ++k) {
    a.scale[k] = k < c ? scale[k] : 0.0;
    a.offset[k] = k < c ? offset[k] : 0.0;
  }
  const long long N = (long long)D * H * W;
  upsample_kernel<<<blocks_for(N, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, src, dst);
  return status_of(cudaGetLastError());
}

int rmrtlb_pack_fields(long long n, int d, const double* rho, const double* u, double rho0, double rho_scale,
                       double u_scale, float* out, void* stream) {
  if (n < 1 || (d != 2 && d != 3) || !rho || !u || !aligned16(out)) return RMRTLB_EINVAL;
  pack_kernel<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, d, rho, u, rho0, rho_scale,
                                                                                u_scale, out);
  return status_of(cudaGetLastError());
}

}  // extern "C"
