// Launch-shape constants of the step kernels, chosen by measurement on
// GB300 (a sweep of the minimum-blocks hint per lattice and storage).  Each may be overridden with -D at build
// time to compare alternatives.
#pragma once

// Minimum resident 128-thread blocks per SM requested from the compiler for
// the two-nodes-per-thread step kernel; this caps registers at
// 65536 / (128 * n), and 1 leaves the count to the compiler.  Measured on
// the full-size workloads with packed FP32 collision (GB/s of the step
// kernel, best setting first):
//   rD2Q9  FP32 12: 6665      16-bit  1: 5066 (12: 4944)
//   rD3Q19 FP32  6: 6842 raw, 6396 central (1: 4941 central)
//          16-bit raw 8: 5448, central 6: 4303 (8: 4088)
//   rD3Q27 FP32  5: 6899 raw, 6312 central (1: 6230 / 4431)
//          16-bit raw 6: 5447, central 5: 4276 (6: 3619)
// FP64 (the correctness path) is left to the compiler.
#ifndef RMRT_X2_MINB_D2Q9_W4
#define RMRT_X2_MINB_D2Q9_W4 12
#endif
#ifndef RMRT_X2_MINB_D2Q9_W2
#define RMRT_X2_MINB_D2Q9_W2 1
#endif
#ifndef RMRT_X2_MINB_D3Q19_W4
#define RMRT_X2_MINB_D3Q19_W4 6
#endif
// FP32 central and central-Hermite bases: the same caps as the raw kernels.
// With the central shift applied as a full second cube of moments they
// spilled 124-168 bytes per thread at these caps; the transported
// second-order correction (subtract_transported) needs no second cube and
// they compile without spills at 80 / 96 registers.
// rD3Q19 central (rechecked with the transported correction, MLUPS): 5
// blocks 44,989 (78 registers), 6: 43,280 (76), 7: 45,032 (72).
#ifndef RMRT_X2_MINB_D3Q19_W4_CENTRAL
#define RMRT_X2_MINB_D3Q19_W4_CENTRAL 7
#endif
#ifndef RMRT_X2_MINB_D3Q19_W2
#define RMRT_X2_MINB_D3Q19_W2 8
#endif
#ifndef RMRT_X2_MINB_D3Q19_W2_CENTRAL
#define RMRT_X2_MINB_D3Q19_W2_CENTRAL 6
#endif
#ifndef RMRT_X2_MINB_D3Q27_W4
#define RMRT_X2_MINB_D3Q27_W4 5
#endif
#ifndef RMRT_X2_MINB_D3Q27_W4_CENTRAL
#define RMRT_X2_MINB_D3Q27_W4_CENTRAL 5
#endif
#ifndef RMRT_X2_MINB_D3Q27_W2
#define RMRT_X2_MINB_D3Q27_W2 6
#endif
#ifndef RMRT_X2_MINB_D3Q27_W2_CENTRAL
#define RMRT_X2_MINB_D3Q27_W2_CENTRAL 5
#endif

// The same hint for the four-nodes-per-thread kernel (16-bit storage).  A
// hint of 1 still changes the compiler's choice (it allows up to 255
// registers; without a hint it keeps fewer).  Measured (MLUPS, FP16 with
// stochastic rounding, best first):
//   rD2Q9           9: 168,330   6: 162,976
//   rD3Q19 raw      1:  78,746   3:  78,659
//   rD3Q19 central  5:  75,435   4:  70,189   3:  69,221
//   rD3Q27 raw      4:  59,177   3:  56,261
//   rD3Q27 central  4:  52,169   3:  51,119   2:  42,802
// (the central bases at these caps since their collision is the raw one
// plus a transported second-order correction, which needs no second cube
// of moments)
#ifndef RMRT_X4_MINB_D2Q9
#define RMRT_X4_MINB_D2Q9 9
#endif
#ifndef RMRT_X4_MINB_D3Q19
#define RMRT_X4_MINB_D3Q19 1
#endif
#ifndef RMRT_X4_MINB_D3Q19_CENTRAL
#define RMRT_X4_MINB_D3Q19_CENTRAL 5
#endif
#ifndef RMRT_X4_MINB_D3Q27
#define RMRT_X4_MINB_D3Q27 4
#endif
#ifndef RMRT_X4_MINB_D3Q27_CENTRAL
#define RMRT_X4_MINB_D3Q27_CENTRAL 4
#endif

namespace rmrt {
// LAT: lattice; BYTES: size of one stored population; CENTRAL: basis.
template <int LAT, int BYTES, bool CENTRAL>
struct Tuning {
  static constexpr int X2_MIN_BLOCKS =
      BYTES == 8 ? 1
      : LAT == 0 ? (BYTES == 4 ? RMRT_X2_MINB_D2Q9_W4 : RMRT_X2_MINB_D2Q9_W2)
      : LAT == 1 ? (BYTES == 4 ? (CENTRAL ? RMRT_X2_MINB_D3Q19_W4_CENTRAL : RMRT_X2_MINB_D3Q19_W4)
                               : (CENTRAL ? RMRT_X2_MINB_D3Q19_W2_CENTRAL : RMRT_X2_MINB_D3Q19_W2))
                 : (BYTES == 4 ? (CENTRAL ? RMRT_X2_MINB_D3Q27_W4_CENTRAL : RMRT_X2_MINB_D3Q27_W4)
                               : (CENTRAL ? RMRT_X2_MINB_D3Q27_W2_CENTRAL : RMRT_X2_MINB_D3Q27_W2));
  static constexpr int X4_MIN_BLOCKS =
      LAT == 0 ? RMRT_X4_MINB_D2Q9
      : LAT == 1 ? (CENTRAL ? RMRT_X4_MINB_D3Q19_CENTRAL : RMRT_X4_MINB_D3Q19)
                 : (CENTRAL ? RMRT_X4_MINB_D3Q27_CENTRAL : RMRT_X4_MINB_D3Q27);
};
}  // namespace rmrt
