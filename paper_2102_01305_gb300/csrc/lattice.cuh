// Lattices, storage types and the fluid kernels' parameter block: the
// definitions the collide-stream kernel is compiled from.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "ibl.h"

namespace ibl {

// ----------------------------------------------------------------- lattices
// Direction order: 0 rest, then pairs (c, -c) so that opp(i) = i + 1 for odd i.
template <int Q> struct Lat;

template <> struct Lat<9> {
  static constexpr int D = 2;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int v[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int v[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    return v[i];
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  // Eq. 5: 4/9 rest, 1/9 axis, 1/36 diagonal
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  // 3 w_i rounded to FP32 values whose discrete moment 2 w3_axis + 4 w3_diag
  // equals 1 exactly (11184811 * 2^-25 and 11184810 * 2^-27)
  __host__ __device__ static constexpr double w3f(int i) {
    return i == 0 ? 0.0 : (i < 5 ? 11184811.0 / 33554432.0 : 11184810.0 / 134217728.0);
  }
};

template <> struct Lat<19> {
  static constexpr int D = 3;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int cz(int i) {
    constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  // 3 w_i rounded to FP32 values whose discrete moment 2 w3_face + 8 w3_edge
  // equals 1 exactly (11184810 * 2^-26 and 11184811 * 2^-27)
  __host__ __device__ static constexpr double w3f(int i) {
    return i == 0 ? 0.0 : (i < 7 ? 11184810.0 / 67108864.0 : 11184811.0 / 134217728.0);
  }
};

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Weight of the odd (momentum-carrying) part of f_eq and of the Guo term,
// 3 w_i.  In FP32 the rounded 1/18, 1/36 (or 1/9, 1/36) break the identity
// sum_i 3 w_i c_i c_i = I by ~1e-8, which makes every collision scale the
// momentum by (1 + omega * 1e-8) - a drift of ~1e-5 after 1000 steps.  The
// FP32 constants below satisfy the identity exactly.
template <int Q, class R> __host__ __device__ constexpr R w3(int i);
template <> __host__ __device__ constexpr float w3<9, float>(int i) { return (float)Lat<9>::w3f(i); }
template <> __host__ __device__ constexpr float w3<19, float>(int i) { return (float)Lat<19>::w3f(i); }
template <> __host__ __device__ constexpr double w3<9, double>(int i) { return 3.0 * Lat<9>::w(i); }
template <> __host__ __device__ constexpr double w3<19, double>(int i) { return 3.0 * Lat<19>::w(i); }

// ----------------------------------------------------------------- storage types
template <class T> struct Store;
template <> struct Store<double> {
  using R = double;
  __device__ static double ld(double v) { return v; }
  __device__ static double st(double v) { return v; }
};
template <> struct Store<float> {
  using R = float;
  __device__ static float ld(float v) { return v; }
  __device__ static float st(float v) { return v; }
};
// FP16 stores (f - w) * 2^8: deviations of a few 1e-3 would otherwise sit
// near FP16's subnormal range (6e-5); the power-of-two scale is exact and
// keeps the largest deviations (|f - w| < 0.5) far below FP16's maximum.
template <> struct Store<__half> {
  using R = float;
  __device__ static float ld(__half v) { return __half2float(v) * (1.0f / 256.0f); }
  __device__ static __half st(float v) { return __float2half_rn(v * 256.0f); }
};
template <> struct Store<__nv_bfloat16> {
  using R = float;
  __device__ static float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};

// ----------------------------------------------------------------- tiles of the IB band
constexpr int TILE_X = 16;
constexpr int TILE_Y = 4;
constexpr int TILE_Z3 = 4;        // 3D tile depth; 2D tiles are 16 x 16 x 1
constexpr int TILE_CELLS = 256;
constexpr int TILE_MARKER_CAP = 512;   // markers whose stencil touches one tile
constexpr int G_MAXNNZ = 192;          // nonzeros per row of the IB system
constexpr int HIST_LEN = 65536;        // force history ring per body
constexpr double FIX_SCALE = 70368744177664.0;   // 2^46: fixed-point scale of the spread sums

// status bits raised on the device
constexpr int ST_DIVERGED = 1;
constexpr int ST_NOTCONV = 2;
constexpr int ST_TIMEOUT = 4;
constexpr int ST_OVERFLOW = 8;     // a band / list / row capacity was exceeded

struct TileGeom {
  int tx, ty, tz;        // tile extents
  int ntx, nty, ntz;     // tiles per axis
  int n_tiles;
};

// Everything the fluid kernels need, passed by value.
template <class R> struct FluidParams {
  int nx, ny, nz;
  long long N;
  int bc[6];
  R u_in[3];
  R rho_out;
  R G[3];
  R omega;     // 1 / tau
  R pref;      // 1 - 1/(2 tau), Guo prefactor (Eq. 8)
  TileGeom tg;
  const int* tile_slot;   // n_tiles, -1 where no band slot; nullptr without markers
  unsigned long long* band_acc;   // [slot][3][TILE_CELLS] fixed-point sum_l w_l D (Eq. 15), cleared on read
  R* band_F;              // [slot][3][TILE_CELLS] IB force density 2 rho du written back (Eq. 26)
  int* status;
};

}  // namespace ibl
