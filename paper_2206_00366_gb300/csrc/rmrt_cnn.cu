// Kernels of the warm-start network (include/rmrtlb_cnn.h): 3 x 3 x 3
// convolution forward and backward, MSE, Adam, input features, trilinear
// upsampling.  BF16 activations and weights, FP32 accumulation.
//
// All three convolutions (forward, input gradient, weight gradient) are
// GEMMs on the tensor cores (tcgen05, rmrt_cnn_tc.cuh).  The weight gradient
// reduces over voxels in a fixed order (per-chunk partials, then a
// fixed-order sum), so results are deterministic.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/rmrtlb.h"
#include "../../include/rmrtlb_cnn.h"
#include "rmrt_cnn_tc.cuh"

namespace {

constexpr int kWeightChunk = 4096;   // voxels per partial sum of the weight gradient
constexpr int kBiasChunk = 1024;     // voxels per partial sum of the bias gradient

struct Vol {
  int n, d, h, w;
  __host__ __device__ long long voxels() const { return (long long)n * d * h * w; }
};

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

// ------------------------------------------------------------------ forward and input gradient
constexpr int kTcThreads = 128;
constexpr uint32_t kWaitLimit = 1u << 26;   // mbarrier polls before a kernel gives up

// Set by a tensor-core kernel whose bounded wait for its MMAs gave up (one
// word per device, in the module's static memory; read and cleared by
// rmrtlb_cnn_check).
__device__ int g_tc_error;

template <int KIN, int NOUT>
struct TcShape {
  static constexpr int KP = KIN < 16 ? 16 : KIN;     // K per tap, padded to the MMA's 16
  static constexpr int NP = NOUT < 16 ? 16 : NOUT;   // N padded to 16 (M = 128 needs N % 16 == 0)
  static constexpr int KC = KP / 8;                  // core matrices along K
  static constexpr int B_TAP = NP * KP * 2;          // bytes of one tap's weights
  // taps per A buffer (one commit per buffer): three for rows of up to 8
  // channels; one for 32-channel rows, whose gather (FP32 rows of 128 bytes
  // in the input gradient) is the bound and wants the occupancy instead
  // (measured, 32 -> 32 input gradient: 608 us with one, 819 us with three)
  static constexpr int GROUP = KIN >= 32 ? 1 : 3;
  static constexpr int A_TAP = 128 * KP * 2;         // bytes of one tap's A tile
  static constexpr int A_BUF = GROUP * A_TAP;        // bytes of one A buffer
  static constexpr int SMEM = 27 * B_TAP + 2 * A_BUF + 64;
};

// See rmrt_cnn_tc.cuh.  MODE 0: forward of a layer with cin = KIN, cout =
// NOUT (in: BF16 x; out: z = acc + bias in FP32 and a = silu(z) or z in
// BF16).  MODE 1: input gradient of a layer with cin = NOUT, cout = KIN (in:
// FP32 dy, rounded to BF16; out: dx = acc * silu'(zin) or acc, FP32).
template <int KIN, int NOUT, int MODE>
__global__ void __launch_bounds__(kTcThreads) conv_tc_kernel(Vol g, const void* __restrict__ in,
                                                             const uint16_t* __restrict__ wt,
                                                             const float* __restrict__ bias,
                                                             const float* __restrict__ zin, int apply_silu,
                                                             float* __restrict__ zout, uint16_t* __restrict__ aout) {
  using S = TcShape<KIN, NOUT>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int s_ok;
  uint8_t* Bs = smem;
  uint8_t* As = smem + 27 * S::B_TAP;
  uint64_t* bar = reinterpret_cast<uint64_t*>(As + 2 * S::A_BUF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;

  // weights of every tap, B_t[n][k] K-major in 8 x 16-byte core matrices
  for (int i = tid; i < 27 * S::NP * S::KP; i += kTcThreads) {
    const int t = i / (S::NP * S::KP), rem = i % (S::NP * S::KP), n = rem / S::KP, k = rem % S::KP;
    uint16_t val = 0;
    if (n < NOUT && k < KIN)
      val = MODE == 0 ? wt[(size_t(t) * KIN + k) * NOUT + n] : wt[(size_t(t) * NOUT + n) * KIN + k];
    *reinterpret_cast<uint16_t*>(Bs + t * S::B_TAP + ((n >> 3) * S::KC + (k >> 3)) * 128 + (n & 7) * 16 +
                                 (k & 7) * 2) = val;
  }
  if (warp == 0) tc::tmem_alloc(tslot, 32);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  const uint32_t idesc = tc::idesc_bf16(S::NP);
  const uint32_t lane_base = uint32_t(warp * 32) << 16;

  const long long V = g.voxels();
  const long long tiles = (V + 127) / 128;
  uint32_t T = 0;   // tap groups issued by this CTA (selects the A buffer and the barrier phase)
  bool ok = true;
  // raw neighbour row of one tap: BF16 (MODE 0) or FP32 (MODE 1) values
  using Raw = typename std::conditional<MODE == 0, uint4, float4>::type;
  constexpr int NRAW = MODE == 0 ? KIN / 8 : KIN / 4;
  constexpr int NRAW1 = NRAW > 0 ? NRAW : 1;
  auto load_row = [&](const VoxCoord& c, bool valid, int t, Raw (&raw)[NRAW1], bool& present) {
    present = false;
    if (!valid) return;
    const int dz = t / 9 - 1, dyo = (t / 3) % 3 - 1, dxo = t % 3 - 1;
    const long long nb = MODE == 0 ? neighbour(c, dz, dyo, dxo, g) : neighbour(c, -dz, -dyo, -dxo, g);
    if (nb < 0) return;
    present = true;
    if constexpr (MODE == 0) {
      const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(in) + nb * KIN);
#pragma unroll
      for (int q = 0; q < NRAW; ++q) raw[q] = __ldg(src + q);
    } else {
      const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(in) + nb * KIN);
#pragma unroll
      for (int q = 0; q < NRAW; ++q) raw[q] = __ldg(src + q);
    }
  };
  for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const long long v = tile * 128 + tid;
    const bool valid = v < V;
    const VoxCoord c = coord_of(valid ? v : 0, g);
    Raw raw[S::GROUP][NRAW1];
    bool present[S::GROUP];
    // the rows of group 0; the rows of group k + 1 are loaded while group k is issued
#pragma unroll
    for (int gg = 0; gg < S::GROUP; ++gg) load_row(c, valid, gg, raw[gg], present[gg]);
    for (int t0 = 0; t0 < 27; t0 += S::GROUP, ++T) {
      const int b = int(T & 1);
      // buffer b is free once the MMAs of group T - 2 have completed
      if (tid == 0) s_ok = T < 2 ? 1 : int(tc::mbar_wait(&bar[b], ((T - 2) >> 1) & 1, kWaitLimit));
      __syncthreads();
      if (!s_ok) { ok = false; break; }
      uint8_t* Ab = As + b * S::A_BUF;
#pragma unroll
      for (int gg = 0; gg < S::GROUP; ++gg) {
        uint4 row[S::KC];
#pragma unroll
        for (int q = 0; q < S::KC; ++q) row[q] = make_uint4(0, 0, 0, 0);
        if (present[gg]) {
          if constexpr (MODE == 0) {
#pragma unroll
            for (int q = 0; q < NRAW; ++q) row[q] = raw[gg][q];
          } else {
            uint32_t pk[S::KP / 2];
#pragma unroll
            for (int q = 0; q < S::KP / 2; ++q) pk[q] = 0;
#pragma unroll
            for (int q = 0; q < NRAW; ++q) {
              pk[2 * q] = uint32_t(f2bf(raw[gg][q].x)) | (uint32_t(f2bf(raw[gg][q].y)) << 16);
              pk[2 * q + 1] = uint32_t(f2bf(raw[gg][q].z)) | (uint32_t(f2bf(raw[gg][q].w)) << 16);
            }
#pragma unroll
            for (int q = 0; q < S::KC; ++q)
              row[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
          }
        }
#pragma unroll
        for (int q = 0; q < S::KC; ++q)
          *reinterpret_cast<uint4*>(Ab + gg * S::A_TAP + ((tid >> 3) * S::KC + q) * 128 + (tid & 7) * 16) = row[q];
      }
      if (t0 + S::GROUP < 27) {
#pragma unroll
        for (int gg = 0; gg < S::GROUP; ++gg) load_row(c, valid, t0 + S::GROUP + gg, raw[gg], present[gg]);
      }
      tc::fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after();
#pragma unroll
        for (int gg = 0; gg < S::GROUP; ++gg) {
          const int t = t0 + gg;
#pragma unroll
          for (int kk = 0; kk < S::KP / 16; ++kk) {
            const uint64_t ad = tc::smem_desc(tc::smem_u32(Ab + gg * S::A_TAP) + kk * 256, 128, S::KC * 128);
            const uint64_t bd = tc::smem_desc(tc::smem_u32(Bs + t * S::B_TAP) + kk * 256, 128, S::KC * 128);
            tc::mma_bf16(taddr, ad, bd, idesc, (t > 0 || kk > 0) ? 1u : 0u);
          }
        }
        tc::mma_commit(&bar[b]);
      }
    }
    if (!ok) break;
    // the last commit covers every MMA issued before it
    if (tid == 0) s_ok = int(tc::mbar_wait(&bar[(T - 1) & 1], ((T - 1) >> 1) & 1, kWaitLimit));
    __syncthreads();
    if (!s_ok) { ok = false; break; }
    tc::fence_after();
    float acc[32];
    tc::tmem_ld16(taddr + lane_base, *reinterpret_cast<float(*)[16]>(acc));
    if constexpr (S::NP == 32) tc::tmem_ld16(taddr + lane_base + 16, *reinterpret_cast<float(*)[16]>(acc + 16));
    tc::fence_before();
    if (valid) {
      if constexpr (MODE == 0) {
#pragma unroll
        for (int n = 0; n < NOUT; ++n) acc[n] += bias[n];
        if (zout) {
          float4* zo = reinterpret_cast<float4*>(zout + v * NOUT);
#pragma unroll
          for (int q = 0; q < NOUT / 4; ++q) zo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
        if (aout) {
          uint32_t* ao = reinterpret_cast<uint32_t*>(aout + v * NOUT);
#pragma unroll
          for (int q = 0; q < NOUT / 2; ++q) {
            float p0 = acc[2 * q], p1 = acc[2 * q + 1];
            if (apply_silu) {
              p0 *= sigm(p0);
              p1 *= sigm(p1);
            }
            ao[q] = uint32_t(f2bf(p0)) | (uint32_t(f2bf(p1)) << 16);
          }
        }
      } else {
        if (zin) {
          // the pre-activation row in 16-byte loads (z_in is 16-byte aligned, NOUT a multiple of 4)
          const float4* zr = reinterpret_cast<const float4*>(zin + v * NOUT);
#pragma unroll
          for (int q4 = 0; q4 < NOUT / 4; ++q4) {
            const float4 z4 = zr[q4];
            const float zs[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float zz = zs[e], sg = sigm(zz);
              acc[4 * q4 + e] *= sg * (1.0f + zz * (1.0f - sg));
            }
          }
        }
        float4* dx = reinterpret_cast<float4*>(zout + v * NOUT);
#pragma unroll
        for (int q = 0; q < NOUT / 4; ++q) dx[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
      }
    }
  }
  if (!ok && tid == 0) atomicExch(&g_tc_error, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

// ------------------------------------------------------------------ forward, fed by the tensor-memory accelerator
// Output tiles are boxes of BW x BH voxels of one (image, z) plane, BW * BH
// = 128 = the MMA's M.  For each of the 27 taps the tensor-memory
// accelerator copies the box shifted by the tap from the channels-last
// input straight into shared memory.  32 channels: one copy of 128 rows x
// 64 bytes with the 64-byte swizzle, which is the MMA's K-major 64-byte
// swizzled layout (8-row atoms of 512 bytes; the second K step of 16
// channels starts 32 bytes into the row).  8 channels: one copy of 128 rows
// x 16 bytes, the canonical no-swizzle K-major layout (8 x 16-byte core
// matrices stacked along M, SBO = 128 bytes), K 8..15 read from a zero
// block (LBO = its distance).  The copy engine moves a box row by row, so
// wide rows (one 64-byte row per voxel rather than four 16-byte ones) keep
// it off the critical path.  Out-of-range
// coordinates read as zero, which is the convolution's zero padding, so no
// thread gathers anything.  Warp roles (192 threads): warp 4 lane 0 issues
// the copies into a ring of STAGES buffers of GROUP taps each, warp 5 lane 0
// issues the MMAs (a buffer is free again once its MMAs complete: one
// tcgen05.commit per buffer, since a commit per tap costs more than the tap),
// and warps 0-3 read the accumulator (one tensor-memory lane per thread)
// while the next tile accumulates into the second of two accumulators.
// Every wait is bounded; a give-up raises the block's abort flag, the copy
// warp waits for its copies still in flight and the MMA warp for its last
// MMAs, and the kernel records the condition for rmrtlb_cnn_check.
// Buffers in the copy ring and taps per buffer (a divisor of 27: the MMAs of
// one buffer are committed once, and a commit is not free); overridable with
// -D to compare alternatives.  Measured on GB300 (4 x 32 x 64 x 64 voxels,
// microseconds for 8->32 / 32->32 / 32->4): 1 tap x 6 buffers 150 / 185 /
// 167; 3 x 2: 124 / 141 / 97; 3 x 3: 123 / 128 / 95; 9 x 2: 123 / 126 / 72.
#ifndef RMRT_TMA_STAGES_K8
#define RMRT_TMA_STAGES_K8 2
#endif
#ifndef RMRT_TMA_STAGES_K32
#define RMRT_TMA_STAGES_K32 2
#endif
#ifndef RMRT_TMA_GROUP_K8
#define RMRT_TMA_GROUP_K8 9
#endif
#ifndef RMRT_TMA_GROUP_K32
#define RMRT_TMA_GROUP_K32 9
#endif
template <int KIN, int NOUT>
struct TmaShape {
  static constexpr int KP = KIN < 16 ? 16 : KIN;      // K per tap, padded to the MMA's 16
  static constexpr int NP = NOUT < 16 ? 16 : NOUT;
  static constexpr int KC = KP / 8;                   // 16-byte chunks of K
  // 32 channels: one copy per tap of 128 rows x 64 bytes, 64-byte swizzle;
  // 8 channels (or 4 padded to 8 in the tensor): one copy of 128 rows x 16
  // bytes (no swizzle) plus a zero block for K 8..15
  static constexpr bool SW64 = KIN == 32;
  static constexpr int LOADED = SW64 ? 1 : (KIN + 7) / 8;   // copies per tap
  static constexpr int CHUNK = SW64 ? 128 * 64 : 128 * 16;
  static constexpr int TAP = LOADED * CHUNK;          // bytes of one tap's A tile
  static constexpr int GROUP = KIN <= 8 ? RMRT_TMA_GROUP_K8 : RMRT_TMA_GROUP_K32;   // taps per buffer
  static constexpr int STAGE = GROUP * TAP;
  static constexpr int STAGES = KIN <= 8 ? RMRT_TMA_STAGES_K8 : RMRT_TMA_STAGES_K32;
  static_assert(27 % GROUP == 0, "taps per buffer must divide 27");
  static constexpr int B_TAP = NP * KP * 2;
  static constexpr int OFF_B = STAGES * STAGE;
  static constexpr int OFF_ZERO = OFF_B + 27 * B_TAP;
  static constexpr int ZERO = (!SW64 && LOADED < KC) ? CHUNK : 0;
  static constexpr int OFF_BAR = OFF_ZERO + ZERO;
  static constexpr int NBAR = 2 * STAGES + 4;
  static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16 + 1024;   // + room to align the base to 1024
};
constexpr int kTmaThreads = 192;
constexpr uint32_t kTmaWaitLimit = 1u << 22;   // polls before a role of the copy-fed kernel gives up

// Bounded wait that also gives up as soon as another role raised `abort`.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
  for (uint32_t i = 0; i < kTmaWaitLimit; i += 64) {
    if (tc::mbar_wait(bar, parity, 64)) return true;
    if (*abort) return false;
  }
  return false;
}

struct TileAt {
  int n, z, y0, x0;
};
__device__ __forceinline__ TileAt tile_at(long long tile, const Vol& g, int bw, int bh, int tx_n, int ty_n) {
  TileAt t;
  t.x0 = int(tile % tx_n) * bw;
  long long r = tile / tx_n;
  t.y0 = int(r % ty_n) * bh;
  r /= ty_n;
  t.z = int(r % g.d);
  t.n = int(r / g.d);
  return t;
}

// MODE 0: forward (in: BF16 x; out: z = acc + bias in FP32 and a = silu(z)
// or z in BF16).  MODE 1: input gradient of a layer with cin = NOUT, cout =
// KIN (in: dy rounded to BF16 beforehand; taps mirrored, weights read as
// w[t, n, k]; out: dx = acc * silu'(zin) or acc, FP32).
template <int KIN, int NOUT, int MODE>
__global__ void __launch_bounds__(kTmaThreads) conv_tma_kernel(const __grid_constant__ CUtensorMap tmap, Vol g,
                                                               int bw, int bh, const uint16_t* __restrict__ wt,
                                                               const float* __restrict__ bias, int apply_silu,
                                                               const float* __restrict__ zin,
                                                               float* __restrict__ zout, uint16_t* __restrict__ aout) {
  using S = TmaShape<KIN, NOUT>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* As = smem;
  uint8_t* Bs = smem + S::OFF_B;
  uint8_t* Zs = smem + S::OFF_ZERO;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::OFF_BAR);
  uint64_t* empty = full + S::STAGES;
  uint64_t* accf = empty + S::STAGES;    // accumulator a written (the MMAs of a tile complete)
  uint64_t* acce = accf + 2;             // accumulator a read out by the four epilogue warps
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights of every tap, B_t[n][k] K-major in 8 x 16-byte core matrices; the zero block
  for (int i = tid; i < 27 * S::NP * S::KP; i += kTmaThreads) {
    const int t = i / (S::NP * S::KP), rem = i % (S::NP * S::KP), n = rem / S::KP, k = rem % S::KP;
    uint16_t val = 0;
    if (n < NOUT && k < KIN)
      val = MODE == 0 ? wt[(size_t(t) * KIN + k) * NOUT + n] : wt[(size_t(t) * NOUT + n) * KIN + k];
    *reinterpret_cast<uint16_t*>(Bs + t * S::B_TAP + ((n >> 3) * S::KC + (k >> 3)) * 128 + (n & 7) * 16 +
                                 (k & 7) * 2) = val;
  }
  for (int i = tid; i < S::ZERO / 16; i += kTmaThreads) reinterpret_cast<uint4*>(Zs)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 5) tc::tmem_alloc(tslot, 64);
  if (tid == 0) {
    for (int k = 0; k < S::STAGES; ++k) {
      tc::mbar_init(&full[k], 1);
      tc::mbar_init(&empty[k], 1);
    }
    tc::mbar_init(&accf[0], 1);
    tc::mbar_init(&accf[1], 1);
    tc::mbar_init(&acce[0], 4);
    tc::mbar_init(&acce[1], 4);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  const int tx_n = (g.w + bw - 1) / bw, ty_n = (g.h + bh - 1) / bh;
  const long long tiles = (long long)g.n * g.d * ty_n * tx_n;

  if (warp == 4) {
    if (lane == 0) {                       // copies
      uint32_t it = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const TileAt p = tile_at(tile, g, bw, bh, tx_n, ty_n);
        for (int t0 = 0; t0 < 27; t0 += S::GROUP) {
          const int st = int(it % S::STAGES);
          const uint32_t round = it / S::STAGES;
          if (round > 0 && !mbar_wait_or_abort(&empty[st], (round - 1) & 1, abort)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&full[st], S::STAGE);
#pragma unroll
          for (int g2 = 0; g2 < S::GROUP; ++g2) {
            const int t = t0 + g2, sg = MODE == 0 ? 1 : -1;   // the input gradient reads v - tap
            const int dz = sg * (t / 9 - 1), dy = sg * ((t / 3) % 3 - 1), dx = sg * (t % 3 - 1);
#pragma unroll
            for (int c = 0; c < S::LOADED; ++c)
              tc::tma_load_5d(As + st * S::STAGE + g2 * S::TAP + c * S::CHUNK, &tmap, &full[st],
                              (S::SW64 ? 32 : 8) * c, p.x0 + dx, p.y0 + dy, p.z + dz, p.n);
          }
          ++it;
        }
      }
      if (!ok) {
        *abort = 1;
        atomicExch(&g_tc_error, 1);
      }
      // no copy may still be writing shared memory when the block exits
      for (uint32_t k = it > uint32_t(S::STAGES) ? it - S::STAGES : 0; k < it; ++k)
        tc::mbar_wait(&full[k % S::STAGES], (k / S::STAGES) & 1, kTmaWaitLimit);
    }
  } else if (warp == 5) {
    if (lane == 0) {                       // MMAs
      const uint32_t idesc = tc::idesc_bf16(S::NP);
      uint32_t it = 0, j = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++j) {
        const uint32_t a = j & 1;
        if (j >= 2 && !mbar_wait_or_abort(&acce[a], ((j >> 1) - 1) & 1, abort)) {
          ok = false;
          break;
        }
        tc::fence_after();
        for (int t0 = 0; t0 < 27; t0 += S::GROUP) {
          const int st = int(it % S::STAGES);
          if (!mbar_wait_or_abort(&full[st], (it / S::STAGES) & 1, abort)) {
            ok = false;
            break;
          }
          tc::fence_after();
#pragma unroll
          for (int g2 = 0; g2 < S::GROUP; ++g2) {
            const int t = t0 + g2;
            const uint32_t abase = tc::smem_u32(As + st * S::STAGE + g2 * S::TAP);
#pragma unroll
            for (int kk = 0; kk < S::KP / 16; ++kk) {
              uint64_t ad;
              if constexpr (S::SW64) {
                ad = tc::smem_desc_sw64(abase + 32 * kk, 512);
              } else {
                const uint32_t a0 = abase + 2 * kk * S::CHUNK;
                const uint32_t lbo = S::ZERO ? tc::smem_u32(Zs) - a0 : uint32_t(S::CHUNK);
                ad = tc::smem_desc(a0, lbo, 128);
              }
              const uint64_t bd = tc::smem_desc(tc::smem_u32(Bs + t * S::B_TAP) + kk * 256, 128, S::KC * 128);
              tc::mma_bf16(taddr + a * 32, ad, bd, idesc, (t > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(&empty[st]);      // the buffer is free once these MMAs have read it
          ++it;
        }
        if (ok) tc::mma_commit(&accf[a]);
      }
      if (!ok) {
        *abort = 1;
        atomicExch(&g_tc_error, 1);
      }
      // the last MMAs must have completed before the accumulators are released
      if (it > 0) tc::mbar_wait(&empty[(it - 1) % S::STAGES], ((it - 1) / S::STAGES) & 1, kTmaWaitLimit);
    }
  } else {                                 // epilogue: warps 0-3, thread = row = tensor-memory lane
    uint32_t j = 0;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++j) {
      const uint32_t a = j & 1;
      int ok = 1;
      if (lane == 0) ok = int(mbar_wait_or_abort(&accf[a], (j >> 1) & 1, abort));
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          *abort = 1;
          atomicExch(&g_tc_error, 1);
        }
        break;
      }
      tc::fence_after();
      float acc[32];
      const uint32_t ta = taddr + (uint32_t(warp * 32) << 16) + a * 32;
      tc::tmem_ld16(ta, *reinterpret_cast<float(*)[16]>(acc));
      if constexpr (S::NP == 32) tc::tmem_ld16(ta + 16, *reinterpret_cast<float(*)[16]>(acc + 16));
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[a]);
      const TileAt p = tile_at(tile, g, bw, bh, tx_n, ty_n);
      const int y = p.y0 + tid / bw, x = p.x0 + tid % bw;
      if (MODE == 1 && y < g.h && x < g.w) {
        const long long v = (((long long)p.n * g.d + p.z) * g.h + y) * g.w + x;
        if (zin) {
          // the pre-activation row in 16-byte loads (z_in is 16-byte aligned, NOUT a multiple of 4)
          const float4* zr = reinterpret_cast<const float4*>(zin + v * NOUT);
#pragma unroll
          for (int q4 = 0; q4 < NOUT / 4; ++q4) {
            const float4 z4 = zr[q4];
            const float zs[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float zz = zs[e], sgm = sigm(zz);
              acc[4 * q4 + e] *= sgm * (1.0f + zz * (1.0f - sgm));
            }
          }
        }
        float4* dxo = reinterpret_cast<float4*>(zout + v * NOUT);
#pragma unroll
        for (int q = 0; q < NOUT / 4; ++q)
          dxo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
      } else if (MODE == 0 && y < g.h && x < g.w) {
        const long long v = (((long long)p.n * g.d + p.z) * g.h + y) * g.w + x;
#pragma unroll
        for (int n = 0; n < NOUT; ++n) acc[n] += bias[n];
        if (zout) {
          float4* zo = reinterpret_cast<float4*>(zout + v * NOUT);
#pragma unroll
          for (int q = 0; q < NOUT / 4; ++q)
            zo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
        if (aout) {
          uint32_t* ao = reinterpret_cast<uint32_t*>(aout + v * NOUT);
#pragma unroll
          for (int q = 0; q < NOUT / 2; ++q) {
            float p0 = acc[2 * q], p1 = acc[2 * q + 1];
            if (apply_silu) {
              p0 *= sigm(p0);
              p1 *= sigm(p1);
            }
            ao[q] = uint32_t(f2bf(p0)) | (uint32_t(f2bf(p1)) << 16);
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 5) {
    tc::fence_after();
    tc::tmem_dealloc(taddr, 64);
  }
}

// ------------------------------------------------------------------ backward weight
// Weight gradient on the tensor cores: per tap group (TPG taps, M = TPG x
// CIN = 128 rows (tap, ci)), per chunk of kWeightChunk voxels,
//   D[(t, ci), co] = sum_v x[v + tap_t, ci] dy[v, co],
// a GEMM with K = voxels.  Both operands are staged MN-major (the voxel a
// thread gathers gives a contiguous run of ci, resp. co): core matrices of 8
// voxels (K) x 16 bytes (8 channels), K tiles of 128 voxels, two buffers.
// The chunk's partial sums go to part[(c * 27 + t) * CIN * COUT + ci * COUT
// + co] like the FP32-pipe kernel's; sum_chunks_kernel adds the chunks in a
// fixed order.  For MN-major operands without swizzling the leading byte
// offset is the stride between core matrices along K and the stride byte
// offset the one along M (N).
constexpr int kWgKT = 128;   // voxels per K tile

template <int CIN, int COUT>
struct WgShape {
  static constexpr int TPG = 128 / CIN;                 // taps per group
  static constexpr int GROUPS = (27 + TPG - 1) / TPG;
  static constexpr int NP = COUT < 16 ? 16 : COUT;
  static constexpr int A_BUF = 128 * kWgKT * 2;         // M x K tile, bytes
  static constexpr int B_BUF = NP * kWgKT * 2;
  static constexpr int SMEM = 2 * (A_BUF + B_BUF) + 64;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kTcThreads) conv_wgrad_tc_kernel(Vol g, const uint16_t* __restrict__ x,
                                                                   const float* __restrict__ dy,
                                                                   float* __restrict__ part) {
  using S = WgShape<CIN, COUT>;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int s_ok;
  uint8_t* As = smem;
  uint8_t* Bs = smem + 2 * S::A_BUF;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + 2 * S::B_BUF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int chunk = blockIdx.x, group = blockIdx.y;
  if (warp == 0) tc::tmem_alloc(tslot, 32);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  constexpr uint32_t idesc = tc::idesc_bf16(S::NP, true);
  // core strides: along M/N 128 bytes, along K (groups of 8 voxels) 16 (resp. NP / 8) cores
  constexpr uint32_t a_mn = 128, a_k = 16 * 128, b_mn = 128, b_k = (S::NP / 8) * 128;
  const long long V = g.voxels();
  const long long v0 = (long long)chunk * kWeightChunk;
  const long long v1 = v0 + kWeightChunk < V ? v0 + kWeightChunk : V;
  const int ntiles = int((v1 - v0 + kWgKT - 1) / kWgKT);
  bool ok = true;
  for (int kt = 0; kt < ntiles; ++kt) {
    const int b = kt & 1;
    if (tid == 0) s_ok = kt < 2 ? 1 : int(tc::mbar_wait(&bar[b], ((kt - 2) >> 1) & 1, kWaitLimit));
    __syncthreads();
    if (!s_ok) { ok = false; break; }
    const long long v = v0 + (long long)kt * kWgKT + tid;   // this thread's voxel (K index tid)
    const bool valid = v < v1;
    const VoxCoord c = coord_of(valid ? v : 0, g);
    uint8_t* Ab = As + b * S::A_BUF;
    uint8_t* Bb = Bs + b * S::B_BUF;
    const int kg = tid >> 3, kr = tid & 7;
#pragma unroll
    for (int tl = 0; tl < S::TPG; ++tl) {
      const int t = group * S::TPG + tl;
      long long nb = -1;
      if (valid && t < 27) nb = neighbour(c, t / 9 - 1, (t / 3) % 3 - 1, t % 3 - 1, g);
      const uint4* src = reinterpret_cast<const uint4*>(x + (nb < 0 ? 0 : nb) * CIN);
#pragma unroll
      for (int cg = 0; cg < CIN / 8; ++cg) {
        const uint4 val = nb < 0 ? make_uint4(0, 0, 0, 0) : __ldg(src + cg);
        const int mg = tl * (CIN / 8) + cg;
        *reinterpret_cast<uint4*>(Ab + (kg * 16 + mg) * 128 + kr * 16) = val;
      }
    }
    {
      const float* src = dy + (valid ? v : 0) * COUT;
#pragma unroll
      for (int ng = 0; ng < S::NP / 8; ++ng) {
        uint32_t pk[4] = {0, 0, 0, 0};
        if (valid && ng * 8 < COUT) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int co = ng * 8 + 2 * e;
            const float f0 = co < COUT ? src[co] : 0.0f, f1 = co + 1 < COUT ? src[co + 1] : 0.0f;
            pk[e] = uint32_t(f2bf(f0)) | (uint32_t(f2bf(f1)) << 16);
          }
        }
        *reinterpret_cast<uint4*>(Bb + (kg * (S::NP / 8) + ng) * 128 + kr * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < kWgKT / 16; ++kk) {
        const uint32_t aoff = kk * 2 * a_k, boff = kk * 2 * b_k;   // two K core groups per MMA
        const uint64_t ad = tc::smem_desc(tc::smem_u32(Ab) + aoff, a_k, a_mn);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(Bb) + boff, b_k, b_mn);
        tc::mma_bf16(taddr, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar[b]);
    }
  }
  if (ok && ntiles > 0) {
    if (tid == 0) s_ok = int(tc::mbar_wait(&bar[(ntiles - 1) & 1], ((ntiles - 1) >> 1) & 1, kWaitLimit));
    __syncthreads();
    ok = s_ok != 0;
  }
  if (ok) {
    tc::fence_after();
    float acc[32];
    const uint32_t lane_base = uint32_t(warp * 32) << 16;
    tc::tmem_ld16(taddr + lane_base, *reinterpret_cast<float(*)[16]>(acc));
    if constexpr (S::NP == 32) tc::tmem_ld16(taddr + lane_base + 16, *reinterpret_cast<float(*)[16]>(acc + 16));
    const int m = tid, tl = m / CIN, ci = m % CIN, t = group * S::TPG + tl;
    if (t < 27) {
      float* out = part + (size_t(chunk) * 27 + t) * CIN * COUT + size_t(ci) * COUT;
#pragma unroll
      for (int co = 0; co < COUT; ++co) out[co] = ntiles > 0 ? acc[co] : 0.0f;
    }
  } else if (tid == 0) {
    atomicExch(&g_tc_error, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

// ------------------------------------------------------------------ backward weight, fed by the tensor-memory accelerator
// The same GEMM, D[(t, ci), co] = sum_v x[v + tap_t, ci] dy[v, co], with K =
// voxels taken box by box: a K tile is a BW x BH box of one (image, z)
// plane (the forward kernel's output boxes), and a chunk is kWgTiles
// consecutive boxes.  For every tap of the group the copy engine brings the
// box of x shifted by the tap, and the box of a BF16 copy of dy; both are
// MN-major operands (a voxel's channels are contiguous, voxels run along K).
// 32 channels come as one copy of 128 rows x 64 bytes with the 64-byte
// swizzle (8-voxel atoms of 512 bytes, taps 8 KB apart along M); 8 channels
// as one copy of 128 rows x 16 bytes without swizzle (core matrices of 8
// voxels x 8 channels, 128 bytes apart along K and 2 KB along M).  Rows of
// 64 bytes move four times the data per row the copy engine handles.
// Out-of-range coordinates read as zero: the zero padding, and zero dy on
// the padded voxels of a ragged box.  Warp roles as in the forward kernel:
// warp 4 lane 0 issues the copies into a ring of WG_STAGES buffers, warp 5
// lane 0 the MMAs (M = TPG taps x CIN channels = 128, N = 32 output
// channels, K = 16 voxels each, one commit per buffer), warps 0-3 read the
// accumulator at the end of the chunk.  Every wait is bounded.  With 4
// output channels dy's copy is padded to 8 channels (16-byte rows, no
// swizzle) and the MMA takes N = 16, its second 8-channel core matrix read
// from a zero block (the stride byte offset points there).
#ifndef RMRT_WG_STAGES
#define RMRT_WG_STAGES 2
#endif
constexpr int kWgTiles = 32;                            // boxes (K tiles of 128 voxels) per chunk

template <int CIN, int COUT>
struct WgTmaShape {
  static constexpr bool SW64 = CIN == 32;
  static constexpr bool NARROW = COUT == 4;             // dy padded to 8 channels, N = 16
  static constexpr int NP = NARROW ? 16 : 32;           // MMA N
  static constexpr int TPG = 128 / CIN;                 // taps per group (M = 128)
  static constexpr int GROUPS = (27 + TPG - 1) / TPG;
  static constexpr int A_TAP = 128 * CIN * 2;           // one tap's box of x
  static constexpr int A_BYTES = TPG * A_TAP;           // 32 KB
  static constexpr int B_BYTES = 128 * (NARROW ? 8 : 32) * 2;   // the box of dy
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int STAGES = RMRT_WG_STAGES;
  static constexpr int OFF_ZERO = STAGES * STAGE;
  static constexpr int ZERO = NARROW ? 256 : 0;         // two zero core matrices (channels 8..15)
  static constexpr int OFF_BAR = OFF_ZERO + ZERO;
  static constexpr int NBAR = 2 * STAGES + 1;
  static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16 + 1024;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kTmaThreads) conv_wgrad_tma_kernel(const __grid_constant__ CUtensorMap tx,
                                                                     const __grid_constant__ CUtensorMap tdy, Vol g,
                                                                     int bw, int bh, float* __restrict__ part) {
  using S = WgTmaShape<CIN, COUT>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::OFF_BAR);
  uint64_t* empty = full + S::STAGES;
  uint64_t* accf = empty + S::STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int chunk = blockIdx.x, group = blockIdx.y;
  const int ntap = (group + 1) * S::TPG <= 27 ? S::TPG : 27 - group * S::TPG;   // taps of this group
  // the A blocks of the group's missing taps are never copied: zero them
  // once (they only feed accumulator rows that are not written out)
  for (int st = 0; st < S::STAGES; ++st)
    for (int i = tid; i < (S::TPG - ntap) * S::A_TAP / 16; i += kTmaThreads)
      reinterpret_cast<uint4*>(smem + st * S::STAGE + ntap * S::A_TAP)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < S::ZERO / 16; i += kTmaThreads)
    reinterpret_cast<uint4*>(smem + S::OFF_ZERO)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 5) tc::tmem_alloc(tslot, 32);
  if (tid == 0) {
    for (int k = 0; k < S::STAGES; ++k) {
      tc::mbar_init(&full[k], 1);
      tc::mbar_init(&empty[k], 1);
    }
    tc::mbar_init(&accf[0], 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *tslot;
  const int tx_n = (g.w + bw - 1) / bw, ty_n = (g.h + bh - 1) / bh;
  const long long tiles = (long long)g.n * g.d * ty_n * tx_n;
  const long long k0 = (long long)chunk * kWgTiles;
  const int nk = int(tiles - k0 < kWgTiles ? tiles - k0 : kWgTiles);

  if (warp == 4) {
    if (lane == 0) {                       // copies
      const uint32_t bytes = uint32_t(ntap * S::A_TAP + S::B_BYTES);
      bool ok = true;
      int issued = 0;
      for (int kt = 0; kt < nk; ++kt) {
        const int st = kt % S::STAGES;
        const int round = kt / S::STAGES;
        if (round > 0 && !mbar_wait_or_abort(&empty[st], (round - 1) & 1, abort)) {
          ok = false;
          break;
        }
        const TileAt p = tile_at(k0 + kt, g, bw, bh, tx_n, ty_n);
        uint8_t* base = smem + st * S::STAGE;
        tc::mbar_expect_tx(&full[st], bytes);
        for (int tl = 0; tl < ntap; ++tl) {
          const int t = group * S::TPG + tl;
          const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
          tc::tma_load_5d(base + tl * S::A_TAP, &tx, &full[st], 0, p.x0 + dx, p.y0 + dy, p.z + dz, p.n);
        }
        tc::tma_load_5d(base + S::A_BYTES, &tdy, &full[st], 0, p.x0, p.y0, p.z, p.n);
        ++issued;
      }
      if (!ok) {
        *abort = 1;
        atomicExch(&g_tc_error, 1);
      }
      // no copy may still be writing shared memory when the block exits
      for (int k = issued > S::STAGES ? issued - S::STAGES : 0; k < issued; ++k)
        tc::mbar_wait(&full[k % S::STAGES], (k / S::STAGES) & 1, kTmaWaitLimit);
    }
  } else if (warp == 5) {
    if (lane == 0) {                       // MMAs
      const uint32_t idesc = tc::idesc_bf16(S::NP, true);
      const uint32_t zbase = tc::smem_u32(smem + S::OFF_ZERO);
      bool ok = true;
      int done = 0;
      for (int kt = 0; kt < nk; ++kt) {
        const int st = kt % S::STAGES;
        if (!mbar_wait_or_abort(&full[st], (kt / S::STAGES) & 1, abort)) {
          ok = false;
          break;
        }
        tc::fence_after();
        const uint32_t abase = tc::smem_u32(smem + st * S::STAGE);
        const uint32_t bbase = abase + S::A_BYTES;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {                       // 16 voxels per MMA
          uint64_t ad;
          if constexpr (S::SW64)
            ad = tc::smem_desc_sw64_mn(abase + kk * 1024, S::A_TAP, 512);
          else
            ad = tc::smem_desc(abase + kk * 256, 128, S::A_TAP);
          uint64_t bd;
          if constexpr (S::NARROW)   // channels 0..7 from the copy, 8..15 from the zero block
            bd = tc::smem_desc(bbase + kk * 256, 128, zbase - (bbase + kk * 256));
          else   // N = 32 is one swizzle atom wide: the N-direction stride is never used
            bd = tc::smem_desc_sw64_mn(bbase + kk * 1024, 512, 512);
          tc::mma_bf16(taddr, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
        }
        tc::mma_commit(&empty[st]);
        ++done;
      }
      if (ok && nk > 0) tc::mma_commit(&accf[0]);
      if (!ok) {
        *abort = 1;
        atomicExch(&g_tc_error, 1);
      }
      // the last MMAs must have completed before the accumulator is released
      if (done > 0) tc::mbar_wait(&empty[(done - 1) % S::STAGES], ((done - 1) / S::STAGES) & 1, kTmaWaitLimit);
    }
  } else {                                 // epilogue: warps 0-3, one accumulator row (tap, ci) per thread
    const bool have = nk > 0 && mbar_wait_or_abort(&accf[0], 0, abort);
    if (nk > 0 && !have && lane == 0) atomicExch(&g_tc_error, 1);
    tc::fence_after();
    float acc[32];
    if (have) {
      const uint32_t lane_base = uint32_t(warp * 32) << 16;
      tc::tmem_ld16(taddr + lane_base, *reinterpret_cast<float(*)[16]>(acc));
      if constexpr (S::NP == 32) tc::tmem_ld16(taddr + lane_base + 16, *reinterpret_cast<float(*)[16]>(acc + 16));
    }
    const int m = tid, tl = m / CIN, ci = m % CIN, t = group * S::TPG + tl;
    if (tl < ntap) {
      float* out = part + (size_t(chunk) * 27 + t) * CIN * COUT + size_t(ci) * COUT;
#pragma unroll
      for (int co = 0; co < COUT; ++co) out[co] = have ? acc[co] : 0.0f;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 5) tc::tmem_dealloc(taddr, 32);
}

// Bias gradient partials, bpart[c * COUT + co] = sum of dy[v, co] over the
// kBiasChunk voxels of chunk c, and with BF16 the copy of dy rounded to
// BF16 (nearest even) that the copy-fed kernels read (4 channels padded to
// rows of 8).  256 threads read the
// chunk's dy as consecutive float4 (COUT a multiple of 4 dividing 1024, so a
// thread always meets the same four channels); the 256 / (COUT / 4) partial
// sums of a channel are then added in a fixed order.
template <int COUT, bool BF16>
__global__ void __launch_bounds__(256) bias_grad_kernel(Vol g, const float* __restrict__ dy,
                                                        float* __restrict__ bpart, void* __restrict__ dy16) {
  static_assert(COUT % 4 == 0 && 1024 % COUT == 0, "four channels per float4, fixed per thread");
  __shared__ float4 red[256];
  const int tid = threadIdx.x;
  const long long V = g.voxels();
  const long long v0 = (long long)blockIdx.x * kBiasChunk;
  const long long v1 = v0 + kBiasChunk < V ? v0 + kBiasChunk : V;
  const long long i1 = v1 * (COUT / 4);
  const float4* src = reinterpret_cast<const float4*>(dy);
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 4
  for (long long i = v0 * (COUT / 4) + tid; i < i1; i += 256) {
    const float4 v = src[i];
    acc.x += v.x;
    acc.y += v.y;
    acc.z += v.z;
    acc.w += v.w;
    if constexpr (BF16) {
      const uint32_t lo = uint32_t(f2bf(v.x)) | (uint32_t(f2bf(v.y)) << 16);
      const uint32_t hi = uint32_t(f2bf(v.z)) | (uint32_t(f2bf(v.w)) << 16);
      if constexpr (COUT == 4)   // one voxel: a row of 8 channels, 4..7 zero (16-byte rows for the copy engine)
        static_cast<uint4*>(dy16)[i] = make_uint4(lo, hi, 0u, 0u);
      else
        static_cast<uint2*>(dy16)[i] = make_uint2(lo, hi);
    }
  }
  red[tid] = acc;
  __syncthreads();
  if (tid < COUT / 4) {
    float4 t = red[tid];
    for (int k = tid + COUT / 4; k < 256; k += COUT / 4) {
      t.x += red[k].x;
      t.y += red[k].y;
      t.z += red[k].z;
      t.w += red[k].w;
    }
    reinterpret_cast<float4*>(bpart + size_t(blockIdx.x) * COUT)[tid] = t;
  }
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

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n < 1)
    return 1;
  return n;
}

template <int KIN, int NOUT, int MODE>
int launch_tc(Vol g, const void* in, const uint16_t* w, const float* bias, const float* zin, int silu, float* zout,
              uint16_t* aout, cudaStream_t s) {
  using S = TcShape<KIN, NOUT>;
  // the opt-in to more than 48 KB of shared memory holds per device: set it on every call
  if (cudaFuncSetAttribute(conv_tc_kernel<KIN, NOUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) != cudaSuccess)
    return RMRTLB_ECUDA;
  const long long tiles = (g.voxels() + 127) / 128;
  const long long cap = 3LL * sm_count();
  const unsigned grid = unsigned(tiles < cap ? tiles : cap);
  conv_tc_kernel<KIN, NOUT, MODE><<<grid, kTcThreads, S::SMEM, s>>>(g, in, w, bias, zin, silu, zout, aout);
  return status_of(cudaGetLastError());
}

// cuTensorMapEncodeTiled of the driver, found through the runtime (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Output box of the copy-fed kernel: BW x BH = 128 voxels, BW a power of
// two, BW <= w and BH <= h, the one covering the plane with the fewest
// padded voxels; false when the plane is too small for any (the gathering
// kernel then runs).
bool pick_box(const Vol& g, int& bw, int& bh) {
  bool found = false;
  long long best = 0;
  for (int b = 128; b >= 8; b >>= 1) {
    const int c = 128 / b;
    if (b > g.w || c > g.h) continue;
    const long long cover = (long long)((g.w + b - 1) / b) * b * ((g.h + c - 1) / c) * c;
    if (!found || cover < best) {
      found = true;
      best = cover;
      bw = b;
      bh = c;
    }
  }
  return found;
}

// Tensor map of a channels-last BF16 tensor (c, x, y, z, image) for boxes
// of all 32 channels (64-byte swizzle) or of 8 channels, BW x BH voxels; a
// 4-channel operand is read from a copy padded to 8 channels.
template <int KIN>
bool make_tmap(CUtensorMap* tm, const Vol& g, const uint16_t* x, int bw, int bh) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  constexpr bool sw64 = TmaShape<KIN, 32>::SW64;
  constexpr int C = KIN < 8 ? 8 : KIN;
  const cuuint64_t dims[5] = {cuuint64_t(C), cuuint64_t(g.w), cuuint64_t(g.h), cuuint64_t(g.d), cuuint64_t(g.n)};
  const cuuint64_t row = cuuint64_t(C) * 2;
  const cuuint64_t strides[4] = {row, row * cuuint64_t(g.w), row * cuuint64_t(g.w) * g.h,
                                 row * cuuint64_t(g.w) * g.h * g.d};
  const cuuint32_t box[5] = {sw64 ? 32u : 8u, cuuint32_t(bw), cuuint32_t(bh), 1, 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<uint16_t*>(x), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, sw64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIN, int NOUT, int MODE>
int run_tma(const CUtensorMap& tm, Vol g, int bw, int bh, const uint16_t* w, const float* bias, int silu,
            const float* zin, float* z, uint16_t* a, cudaStream_t s) {
  using S = TmaShape<KIN, NOUT>;
  // the opt-in to more than 48 KB of shared memory holds per device: set it on every call
  if (cudaFuncSetAttribute(conv_tma_kernel<KIN, NOUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) !=
      cudaSuccess)
    return RMRTLB_ECUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_tma_kernel<KIN, NOUT, MODE>, kTmaThreads,
                                                    S::SMEM) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const long long tiles = (long long)g.n * g.d * ((g.h + bh - 1) / bh) * ((g.w + bw - 1) / bw);
  const long long cap = (long long)per_sm * sm_count();
  const unsigned grid = unsigned(tiles < cap ? tiles : cap);
  conv_tma_kernel<KIN, NOUT, MODE><<<grid, kTmaThreads, S::SMEM, s>>>(tm, g, bw, bh, w, bias, silu, zin, z, a);
  return status_of(cudaGetLastError());
}

template <int KIN, int NOUT>
int launch_tma(Vol g, const uint16_t* x, const uint16_t* w, const float* bias, int silu, float* z, uint16_t* a,
               cudaStream_t s) {
  int bw = 0, bh = 0;
  CUtensorMap tm;
  if (!pick_box(g, bw, bh) || !make_tmap<KIN>(&tm, g, x, bw, bh))
    return launch_tc<KIN, NOUT, 0>(g, x, w, bias, nullptr, silu, z, a, s);
  return run_tma<KIN, NOUT, 0>(tm, g, bw, bh, w, bias, silu, nullptr, z, a, s);
}

// FP32 -> BF16 (nearest even), count a multiple of 4.
__global__ void to_bf16_kernel(long long count4, const float4* __restrict__ in, uint2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count4;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 v = in[i];
    out[i] = make_uint2(uint32_t(f2bf(v.x)) | (uint32_t(f2bf(v.y)) << 16),
                        uint32_t(f2bf(v.z)) | (uint32_t(f2bf(v.w)) << 16));
  }
}

// FP32 -> BF16 (nearest even) of a 4-channel tensor into rows of 8
// channels, channels 4..7 zero (16-byte rows for the copy engine).
__global__ void to_bf16_pad8_kernel(long long voxels, const float4* __restrict__ in, uint4* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < voxels;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 v = in[i];
    out[i] = make_uint4(uint32_t(f2bf(v.x)) | (uint32_t(f2bf(v.y)) << 16),
                        uint32_t(f2bf(v.z)) | (uint32_t(f2bf(v.w)) << 16), 0u, 0u);
  }
}

// Scratch of the copy-fed input gradient, on planes that hold a 128-voxel
// box: a BF16 copy of dy (32 channels, or 4 padded to 8), else none.
size_t bwd_data_scratch(const Vol& g, int cout) {
  int bw = 0, bh = 0;
  if ((cout != 32 && cout != 4) || !pick_box(g, bw, bh)) return 0;
  return size_t(g.voxels()) * (cout == 32 ? 32 : 8) * 2;
}

int chunks_of(Vol g) { return int((g.voxels() + kWeightChunk - 1) / kWeightChunk); }
int bias_chunks_of(Vol g) { return int((g.voxels() + kBiasChunk - 1) / kBiasChunk); }

// Scratch of the weight gradient: chunk partials of dw (for the flat
// kWeightChunk-voxel chunks of the gathering kernel or the box chunks of
// the copy-fed one, whichever are more), chunk partials of db, and, where
// the copy-fed kernel runs (32 output channels, planes that hold a box), a
// BF16 copy of dy; every part starts at a 16-byte boundary.
struct WgScratch {
  size_t part, bpart, dy16_off, total;
  long long box_chunks;
};
WgScratch wgrad_scratch(const Vol& g, int cin, int cout) {
  WgScratch w{};
  const long long flat = chunks_of(g);
  int bw = 0, bh = 0;
  const bool copy_fed = (cout == 32 && (cin == 8 || cin == 32)) || (cin == 32 && cout == 4);
  if (copy_fed && pick_box(g, bw, bh)) {
    const long long tiles = (long long)g.n * g.d * ((g.h + bh - 1) / bh) * ((g.w + bw - 1) / bw);
    w.box_chunks = (tiles + kWgTiles - 1) / kWgTiles;
  }
  const long long parts = flat > w.box_chunks ? flat : w.box_chunks;
  w.part = size_t(parts) * 27 * size_t(cin) * cout * sizeof(float);
  w.bpart = size_t(bias_chunks_of(g)) * cout * sizeof(float);
  w.dy16_off = (w.part + w.bpart + 15) / 16 * 16;
  w.total = w.box_chunks > 0 ? w.dy16_off + size_t(g.voxels()) * (cout == 4 ? 8 : 32) * 2 : w.part + w.bpart;
  return w;
}

template <int CIN, int COUT>
int wgrad_tc(Vol g, const uint16_t* x, const float* dy, float* dw, float* db, float* scratch, cudaStream_t s) {
  using S = WgShape<CIN, COUT>;
  // the opt-in to more than 48 KB of shared memory holds per device: set it on every call
  if (cudaFuncSetAttribute(conv_wgrad_tc_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) !=
      cudaSuccess)
    return RMRTLB_ECUDA;
  const int chunks = chunks_of(g), bchunks = bias_chunks_of(g);
  float* part = scratch;
  float* bpart = scratch + wgrad_scratch(g, CIN, COUT).part / sizeof(float);
  conv_wgrad_tc_kernel<CIN, COUT><<<dim3(chunks, S::GROUPS), kTcThreads, S::SMEM, s>>>(g, x, dy, part);
  bias_grad_kernel<COUT, false><<<bchunks, 256, 0, s>>>(g, dy, bpart, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return RMRTLB_ECUDA;
  const int nw = 27 * CIN * COUT;
  sum_chunks_kernel<<<blocks_for(nw, 256), 256, 0, s>>>(part, chunks, size_t(nw), nw, dw);
  sum_chunks_kernel<<<1, 256, 0, s>>>(bpart, bchunks, size_t(COUT), COUT, db);
  return status_of(cudaGetLastError());
}

// The copy-fed weight gradient (32 output channels, or 4 after 32 inputs).
// Returns false, having launched nothing, where it does not apply (no box
// fits the plane, the scratch is short, or a tensor map cannot be made);
// else true with the status in *status.
template <int CIN, int COUT>
bool wgrad_tma(Vol g, const uint16_t* x, const float* dy, float* dw, float* db, char* scratch, size_t scratch_bytes,
               cudaStream_t s, int* status) {
  using S = WgTmaShape<CIN, COUT>;
  const WgScratch w = wgrad_scratch(g, CIN, COUT);
  int bw = 0, bh = 0;
  if (w.box_chunks == 0 || scratch_bytes < w.total || !pick_box(g, bw, bh)) return false;
  uint16_t* dy16 = reinterpret_cast<uint16_t*>(scratch + w.dy16_off);
  CUtensorMap tx, tdy;
  if (!make_tmap<CIN>(&tx, g, x, bw, bh) || !make_tmap<COUT>(&tdy, g, dy16, bw, bh)) return false;
  // the opt-in to more than 48 KB of shared memory holds per device: set it on every call
  if (cudaFuncSetAttribute(conv_wgrad_tma_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           S::SMEM) != cudaSuccess) {
    *status = RMRTLB_ECUDA;
    return true;
  }
  float* part = reinterpret_cast<float*>(scratch);
  float* bpart = reinterpret_cast<float*>(scratch + w.part);
  const int bchunks = bias_chunks_of(g);
  // one pass over dy: the bias partials and the BF16 copy the copies read
  bias_grad_kernel<COUT, true><<<bchunks, 256, 0, s>>>(g, dy, bpart, dy16);
  conv_wgrad_tma_kernel<CIN, COUT><<<dim3(unsigned(w.box_chunks), S::GROUPS), kTmaThreads, S::SMEM, s>>>(
      tx, tdy, g, bw, bh, part);
  if (cudaGetLastError() != cudaSuccess) {
    *status = RMRTLB_ECUDA;
    return true;
  }
  const int nw = 27 * CIN * COUT;
  sum_chunks_kernel<<<blocks_for(nw, 256), 256, 0, s>>>(part, int(w.box_chunks), size_t(nw), nw, dw);
  sum_chunks_kernel<<<1, 256, 0, s>>>(bpart, bchunks, size_t(COUT), COUT, db);
  *status = status_of(cudaGetLastError());
  return true;
}

// An mbarrier that nothing arrives on, waited for with the convolutions'
// bounded polling: the wait gives up after `polls` polls and the give-up
// is recorded in the same error word.
__global__ void wait_selftest_kernel(uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!tc::mbar_wait(&bar, 0, polls)) atomicExch(&g_tc_error, 1);
  }
}

}  // namespace

extern "C" {

int rmrtlb_conv3d_forward(int n, int d, int h, int w, int cin, int cout, const uint16_t* x, const uint16_t* weight,
                          const float* bias, int apply_silu, float* z, uint16_t* a, void* stream) {
  if (!vol_ok(n, d, h, w) || !aligned16(x) || !weight || !bias || (!z && !a)) return RMRTLB_EINVAL;
  if ((z && !aligned16(z)) || (a && (reinterpret_cast<size_t>(a) & 7))) return RMRTLB_EINVAL;
  const Vol g{n, d, h, w};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cin == 8 && cout == 32) return launch_tma<8, 32>(g, x, weight, bias, apply_silu, z, a, s);
  if (cin == 32 && cout == 32) return launch_tma<32, 32>(g, x, weight, bias, apply_silu, z, a, s);
  if (cin == 32 && cout == 4) return launch_tma<32, 4>(g, x, weight, bias, apply_silu, z, a, s);
  return RMRTLB_EINVAL;
}

size_t rmrtlb_conv3d_backward_data_scratch(int n, int d, int h, int w, int cin, int cout) {
  if (!vol_ok(n, d, h, w) || cin != 32) return 0;
  return bwd_data_scratch(Vol{n, d, h, w}, cout);
}

int rmrtlb_conv3d_backward_data(int n, int d, int h, int w, int cin, int cout, const float* dy,
                                const uint16_t* weight, const float* z_in, float* dx, void* scratch,
                                size_t scratch_bytes, void* stream) {
  if (!vol_ok(n, d, h, w) || !aligned16(dy) || !weight || !aligned16(dx) || (z_in && !aligned16(z_in)))
    return RMRTLB_EINVAL;
  const Vol g{n, d, h, w};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cin == 32 && cout == 32) {
    const size_t need = bwd_data_scratch(g, cout);
    int bw = 0, bh = 0;
    CUtensorMap tm;
    uint16_t* dy16 = static_cast<uint16_t*>(scratch);
    if (need && scratch && aligned16(scratch) && scratch_bytes >= need && pick_box(g, bw, bh) &&
        make_tmap<32>(&tm, g, dy16, bw, bh)) {
      const long long count4 = g.voxels() * 32 / 4;
      const unsigned grid = blocks_for(count4, 256) < 8192u ? blocks_for(count4, 256) : 8192u;
      to_bf16_kernel<<<grid, 256, 0, s>>>(count4, reinterpret_cast<const float4*>(dy), reinterpret_cast<uint2*>(dy16));
      if (cudaGetLastError() != cudaSuccess) return RMRTLB_ECUDA;
      return run_tma<32, 32, 1>(tm, g, bw, bh, weight, nullptr, 0, z_in, dx, nullptr, s);
    }
    return launch_tc<32, 32, 1>(g, dy, weight, nullptr, z_in, 0, dx, nullptr, s);
  }
  if (cin == 32 && cout == 4) {
    const size_t need = bwd_data_scratch(g, cout);
    int bw = 0, bh = 0;
    CUtensorMap tm;
    uint16_t* dy16 = static_cast<uint16_t*>(scratch);
    if (need && scratch && aligned16(scratch) && scratch_bytes >= need && pick_box(g, bw, bh) &&
        make_tmap<4>(&tm, g, dy16, bw, bh)) {
      const long long v = g.voxels();
      const unsigned grid = blocks_for(v, 256) < 8192u ? blocks_for(v, 256) : 8192u;
      to_bf16_pad8_kernel<<<grid, 256, 0, s>>>(v, reinterpret_cast<const float4*>(dy), reinterpret_cast<uint4*>(dy16));
      if (cudaGetLastError() != cudaSuccess) return RMRTLB_ECUDA;
      return run_tma<4, 32, 1>(tm, g, bw, bh, weight, nullptr, 0, z_in, dx, nullptr, s);
    }
    return launch_tc<4, 32, 1>(g, dy, weight, nullptr, z_in, 0, dx, nullptr, s);
  }
  return RMRTLB_EINVAL;
}

size_t rmrtlb_conv3d_backward_weight_scratch(int n, int d, int h, int w, int cin, int cout) {
  if (!vol_ok(n, d, h, w) || cin < 1 || cout < 1) return 0;
  return wgrad_scratch(Vol{n, d, h, w}, cin, cout).total;
}

int rmrtlb_conv3d_backward_weight(int n, int d, int h, int w, int cin, int cout, const uint16_t* x, const float* dy,
                                  float* dweight, float* dbias, void* scratch, size_t scratch_bytes, void* stream) {
  if (!vol_ok(n, d, h, w) || !aligned16(x) || !aligned16(dy) || !dweight || !dbias || !aligned16(scratch))
    return RMRTLB_EINVAL;
  if (scratch_bytes < rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, cin, cout)) return RMRTLB_ENOMEM;
  const Vol g{n, d, h, w};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* sc = static_cast<float*>(scratch);
  char* raw = static_cast<char*>(scratch);
  int status = RMRTLB_OK;
  if (cin == 8 && cout == 32) {
    if (wgrad_tma<8, 32>(g, x, dy, dweight, dbias, raw, scratch_bytes, s, &status)) return status;
    return wgrad_tc<8, 32>(g, x, dy, dweight, dbias, sc, s);
  }
  if (cin == 32 && cout == 32) {
    if (wgrad_tma<32, 32>(g, x, dy, dweight, dbias, raw, scratch_bytes, s, &status)) return status;
    return wgrad_tc<32, 32>(g, x, dy, dweight, dbias, sc, s);
  }
  if (cin == 32 && cout == 4) {
    if (wgrad_tma<32, 4>(g, x, dy, dweight, dbias, raw, scratch_bytes, s, &status)) return status;
    return wgrad_tc<32, 4>(g, x, dy, dweight, dbias, sc, s);
  }
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

int rmrtlb_cnn_check(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return RMRTLB_ECUDA;
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, g_tc_error, sizeof(int)) != cudaSuccess) return RMRTLB_ECUDA;
  const int zero = 0;
  if (h && cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int)) != cudaSuccess) return RMRTLB_ECUDA;
  return h ? RMRTLB_ETIMEOUT : RMRTLB_OK;
}

int rmrtlb_cnn_wait_selftest(unsigned polls, void* stream) {
  if (polls < 1 || polls > (1u << 20)) return RMRTLB_EINVAL;
  wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(polls);
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
